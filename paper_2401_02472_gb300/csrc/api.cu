// The C ABI: argument checks, host/device staging, choice of form, and the
// reruns that keep results exact when a representation runs out of range.
#include <cuda_runtime.h>

#include <algorithm>
#include <climits>
#include <cmath>
#include <limits>
#include <cstdlib>
#include <cstdio>
#include <cstring>
#include <string>
#include <map>
#include <tuple>
#include <initializer_list>
#include <vector>

#include "common.cuh"
#include "internal.h"

namespace sp {

static thread_local std::string g_last_error;

void set_last_error(const std::string& s) { g_last_error = s; }

sp_status fail(sp_status st, const std::string& what) {
    set_last_error(std::string(sp_status_string(st)) + ": " + what);
    return st;
}

sp_status cuda_fail(cudaError_t e, const char* what) {
    std::string s = std::string(what) + ": " + cudaGetErrorString(e);
    if (e == cudaErrorMemoryAllocation) return fail(SP_ERR_OOM, s);
    return fail(SP_ERR_CUDA, s);
}

static bool is_device_ptr(const void* p) {
    if (!p) return false;
    cudaPointerAttributes at{};
    cudaError_t e = cudaPointerGetAttributes(&at, p);
    if (e != cudaSuccess) {
        cudaGetLastError();
        return false;
    }
    return at.type == cudaMemoryTypeDevice || at.type == cudaMemoryTypeManaged;
}

// Device memory of a GPU other than the current one.  Such buffers are
// refused: the kernels read and write device buffers directly, and without
// peer access that would be an illegal access on a shared GPU.
static bool on_other_device(const void* p) {
    if (!p) return false;
    cudaPointerAttributes at{};
    if (cudaPointerGetAttributes(&at, p) != cudaSuccess) {
        cudaGetLastError();
        return false;
    }
    if (at.type != cudaMemoryTypeDevice) return false;
    int dev = 0;
    if (cudaGetDevice(&dev) != cudaSuccess) {
        cudaGetLastError();
        return false;
    }
    return at.device != dev;
}

static sp_status refuse_other_device(std::initializer_list<const void*> ptrs, const char* call) {
    for (const void* p : ptrs)
        if (on_other_device(p))
            return fail(SP_ERR_INVALID_ARG, std::string(call) + ": a buffer is device memory of another GPU");
    return SP_OK;
}

static sp_status check_device() {
    int dev = 0;
    cudaError_t e = cudaGetDevice(&dev);
    if (e != cudaSuccess) {
        cudaGetLastError();
        return fail(SP_ERR_NO_DEVICE, "no CUDA device");
    }
    int major = 0, minor = 0;
    cudaDeviceGetAttribute(&major, cudaDevAttrComputeCapabilityMajor, dev);
    cudaDeviceGetAttribute(&minor, cudaDevAttrComputeCapabilityMinor, dev);
    if (major != 10 || minor != 3)
        return fail(SP_ERR_NO_DEVICE, "this build targets compute capability 10.3 (sm_103a); device " +
                                          std::to_string(dev) + " is " + std::to_string(major) + "." +
                                          std::to_string(minor));
    static bool pool_set[64] = {false};
    if (dev >= 0 && dev < 64 && !pool_set[dev]) {
        // Keep freed workspace in the stream-ordered pool between calls.
        cudaMemPool_t pool;
        if (cudaDeviceGetDefaultMemPool(&pool, dev) == cudaSuccess) {
            uint64_t keep = UINT64_MAX;
            cudaMemPoolSetAttribute(pool, cudaMemPoolAttrReleaseThreshold, &keep);
        }
        pool_set[dev] = true;
    }
    return SP_OK;
}

// A device copy of `count` int32 from host or device memory (freed by the caller).
static sp_status stage_in(const int32_t* src, int64_t count, cudaStream_t st, int32_t** out) {
    *out = nullptr;
    if (count <= 0) return SP_OK;
    SP_CUDA(cudaMallocAsync((void**)out, sizeof(int32_t) * (size_t)count, st));
    cudaMemcpyKind kind = is_device_ptr(src) ? cudaMemcpyDeviceToDevice : cudaMemcpyHostToDevice;
    cudaError_t e = cudaMemcpyAsync(*out, src, sizeof(int32_t) * (size_t)count, kind, st);
    if (e != cudaSuccess) {
        cudaFreeAsync(*out, st);
        *out = nullptr;
        return cuda_fail(e, "copying input");
    }
    return SP_OK;
}

__global__ void check_sources_kernel(const int32_t* s, int32_t nsrc, int32_t n, int* bad) {
    for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < nsrc; i += gridDim.x * blockDim.x)
        if (s[i] < 0 || s[i] >= n) atomicMin(bad, i);
}

static sp_status check_sources(const int32_t* d_src, int32_t nsrc, int32_t n, cudaStream_t st) {
    if (nsrc <= 0) return SP_OK;
    int* d_bad = nullptr;
    SP_CUDA(cudaMallocAsync((void**)&d_bad, sizeof(int), st));
    int h_bad = INT32_MAX;
    cudaError_t e = cudaMemcpyAsync(d_bad, &h_bad, sizeof(int), cudaMemcpyHostToDevice, st);
    if (e == cudaSuccess) {
        check_sources_kernel<<<std::min(1024, (nsrc + 255) / 256), 256, 0, st>>>(d_src, nsrc, n, d_bad);
        e = cudaGetLastError();
    }
    if (e == cudaSuccess) e = cudaMemcpyAsync(&h_bad, d_bad, sizeof(int), cudaMemcpyDeviceToHost, st);
    cudaFreeAsync(d_bad, st);
    if (e == cudaSuccess) e = cudaStreamSynchronize(st);
    if (e != cudaSuccess) return cuda_fail(e, "checking sources");
    if (h_bad != INT32_MAX)
        return fail(SP_ERR_INVALID_ARG, "source " + std::to_string(h_bad) + " is not a vertex id in [0, n)");
    return SP_OK;
}

std::string barrier_diagnostic(const Ctl& h, int grid) {
    int lo = INT32_MAX, hi = INT32_MIN, nlo = 0;
    for (int b = 0; b < grid && b < 1024; ++b) {
        int p = h.block_phase[b];
        if (p < lo) { lo = p; nlo = 0; }
        if (p == lo) ++nlo;
        hi = std::max(hi, p);
    }
    return " (timed out at barrier " + std::to_string(h.err_where) + " with " + std::to_string(h.timeout_count) +
           " of " + std::to_string(grid) + " blocks arrived; blocks' last barriers " + std::to_string(lo) + ".." +
           std::to_string(hi) + ", " + std::to_string(nlo) + " at the lowest)";
}

static sp_status map_device_error(int err, const char* form, const std::string& diag = "") {
    if (err == 0) return SP_OK;
    std::string f = std::string(form) + diag;
    switch (err) {
        case SP_ERR_RANGE: return fail(SP_ERR_RANGE, f + ": a path count or dependency left the FP64 range");
        case SP_ERR_TIMEOUT: return fail(SP_ERR_TIMEOUT, f + ": a grid barrier wait timed out");
        case kErrCapacity:
        case kErrCapEntries:
        case kErrCapHubs:
        case kErrCapLevels: return fail(SP_ERR_TOO_LARGE, f + ": workspace capacity exceeded");
        case kErrSigmaOverflow: return fail(SP_ERR_RANGE, f + ": path counts overflowed");
        case kErrThetaRange32: return fail(SP_ERR_RANGE, f + ": FP32 dependency out of range");
        case kErrCorrupt: return fail(SP_ERR_CUDA, f + ": device state out of range (internal error)");
        case SP_ERR_INVALID_ARG:
            return fail(SP_ERR_INVALID_ARG, f + ": a source in the device array is not a vertex id in [0, n)");
        default: return fail(SP_ERR_CUDA, f + ": device error " + std::to_string(err));
    }
}

static uint64_t bfs_timeout_ns() {
    const char* e = getenv("SP_BARRIER_TIMEOUT_NS");
    return e ? strtoull(e, nullptr, 10) : 20000000000ull;
}

static uint64_t timeout_of(const sp_bc_opts& o) {
    return o.barrier_timeout_ns > 0 ? (uint64_t)o.barrier_timeout_ns : bfs_timeout_ns();
}

// Device bytes one batched launch of this width allocates (default capacities).
size_t batched_workspace_bytes(const Graph* g, int width, bool theta_f32) {
    const size_t n = (size_t)g->n, W = (size_t)width / 32, B = (size_t)width;
    const size_t lcap = std::min<size_t>(n + 2, 16384);
    const size_t ecap = std::min<size_t>(std::max<size_t>(8 * n, 1 << 16), n * std::min(B, lcap));
    const size_t arcs = (size_t)g->knnz();
    const size_t hcap = arcs / 512 * 8 + 1024, segcap = arcs / 1024 + arcs / 512 + 2;
    return 4 * 4 * n * W + 4 * n * W + 4 * n + 8 * n * B + (theta_f32 ? 4 : 8) * n * B + ecap * (4 + 4 * W) +
           hcap * 24 + segcap * B * 8 + 2 * lcap * B * 4 + 3 * (lcap + 2) * 8 + (1 << 20);
}

// Autotuned batch widths, keyed by graph signature (n, nnz, max degree) and
// precision, so that a graph re-created from the same CSR reuses the choice.
static std::mutex g_tune_mu;
// Batched-form choices made by timing: width and bottom-up threshold (a
// value for sp_bc_opts.bottom_up).
struct BatchTune {
    int width;
    int bottom_up;
};
static std::map<std::tuple<int32_t, int64_t, int32_t, int32_t>, BatchTune> g_tuned;

static std::tuple<int32_t, int64_t, int32_t, int32_t> tune_key(const Graph* g, int precision) {
    return std::make_tuple(g->n, g->nnz, g->info.max_degree, (int32_t)precision | (g->directed ? 0x100 : 0));
}

// Representation hints learnt by earlier calls on a graph with the same
// signature: path counts past 64 bits (bit 0), FP32 dependencies out of range
// (bit 1).  They only skip attempts that would fail and be rerun.
static std::map<std::tuple<int32_t, int64_t, int32_t, bool>, int> g_hints;

static int range_hints(const Graph* g) {
    std::lock_guard<std::mutex> lk(g_tune_mu);
    auto it = g_hints.find(std::make_tuple(g->n, g->nnz, g->info.max_degree, g->directed));
    return it == g_hints.end() ? 0 : it->second;
}

static void add_range_hint(const Graph* g, int bit) {
    std::lock_guard<std::mutex> lk(g_tune_mu);
    g_hints[std::make_tuple(g->n, g->nnz, g->info.max_degree, g->directed)] |= bit;
}

static sp_status bc_device(Graph* g, const int32_t* d_src, int32_t nsrc, const sp_bc_opts& o, double* d_bc,
                           sp_bc_stats* stats, cudaStream_t st, double* d_sq = nullptr);
static void absorb_hints(Graph* g);

// Time the batched form on the call's first min(nsrc, 256) sources at each
// width 32 / 64 / 128 / 256 — the same sources for every width — with
// bottom-up discovery off and at n/100 (unless the caller fixed it; graphs
// below 2^18 vertices only off), and keep the pair with the most traversed
// arcs per second of kernel time.
static sp_status autotune_batched(Graph* g, const int32_t* d_src, int32_t nsrc, const sp_bc_opts& o, cudaStream_t st,
                                  BatchTune* out, int* launches) {
    double* scratch = nullptr;
    SP_CUDA(cudaMallocAsync((void**)&scratch, sizeof(double) * (size_t)g->n, st));
    const int32_t sample = std::min<int32_t>(nsrc, 256);
    double best_rate = -1.0;
    BatchTune best{default_batch_width(nsrc), o.bottom_up};
    std::vector<int> bus;
    if (o.bottom_up != 0) bus.push_back(o.bottom_up);
    else {
        bus.push_back(-1);
        if (g->n >= (1 << 18)) bus.push_back(100);
    }
    for (int w : {32, 64, 128, 256}) {
        if (w > sample) break;
        for (int bu : bus) {
            sp_bc_opts t = o;
            t.form = SP_FORM_BATCHED;
            t.batch = w;
            t.bottom_up = bu;
            sp_bc_stats ts;
            sp_status rc = bc_device(g, d_src, sample, t, scratch, &ts, st);
            *launches += ts.launches;
            if (rc != SP_OK) {
                cudaFreeAsync(scratch, st);
                return rc;
            }
            const double rate = ts.kernel_ms > 0 ? (double)ts.traversed_arcs / ts.kernel_ms : 0.0;
            if (rate > best_rate) {
                best_rate = rate;
                best = BatchTune{w, bu};
            }
        }
    }
    cudaFreeAsync(scratch, st);
    *out = best;
    return SP_OK;
}

int default_batch_width(int32_t nsrc) { return nsrc > 32 ? 64 : 32; }

// Plain-form choices made by timing, keyed like the widths: the level-loop
// driver and the bottom-up threshold (a value for sp_bc_opts.bottom_up).
struct PlainTune {
    int driver;
    int bottom_up;
};
static std::map<std::tuple<int32_t, int64_t, int32_t, int32_t>, PlainTune> g_plain_tune;

// Time the plain form on the call's first eight sources: the persistent
// driver with bottom-up discovery off, at n/100 and at n/20 (unless the
// caller fixed the threshold), then the graph driver with the best threshold;
// keep the pair with the most traversed arcs per second of kernel time.
static sp_status autotune_plain(Graph* g, const int32_t* d_src, const sp_bc_opts& o, cudaStream_t st,
                                PlainTune* out, int* launches) {
    double* scratch = nullptr;
    SP_CUDA(cudaMallocAsync((void**)&scratch, sizeof(double) * (size_t)g->n, st));
    double best_rate = -1.0;
    PlainTune best{SP_DRIVER_PERSISTENT, o.bottom_up};
    auto trial = [&](int drv, int bu) -> sp_status {
        sp_bc_opts t = o;
        t.form = SP_FORM_PLAIN;
        t.driver = drv;
        t.bottom_up = bu;
        sp_bc_stats ts;
        sp_status rc = bc_device(g, d_src, 8, t, scratch, &ts, st);
        *launches += ts.launches;
        if (rc != SP_OK) return rc;
        const double rate = ts.kernel_ms > 0 ? (double)ts.traversed_arcs / ts.kernel_ms : 0.0;
        if (rate > best_rate) {
            best_rate = rate;
            best = PlainTune{drv, bu};
        }
        return SP_OK;
    };
    sp_status rc = SP_OK;
    if (o.bottom_up != 0) {
        rc = trial(SP_DRIVER_PERSISTENT, o.bottom_up);
    } else {
        for (int bu : {-1, 100, 20})
            if (rc == SP_OK) rc = trial(SP_DRIVER_PERSISTENT, bu);
    }
    if (rc == SP_OK) rc = trial(SP_DRIVER_GRAPH, best.bottom_up);
    cudaFreeAsync(scratch, st);
    if (rc != SP_OK) return rc;
    *out = best;
    return SP_OK;
}

// Sort key of each source: its hop distances from three landmarks (the three
// vertices of largest degree; distances clamped to 255), then the smallest
// neighbour one hop closer to the first landmark.  Sources with equal
// distances to the hubs through which most shortest paths run sit at the same
// BFS level for most vertices, so batching them in adjacent bit positions
// fills mask words and shares the 32-byte sectors of the per-(vertex, source)
// rows the kernels gather.
__global__ void source_keys_kernel(const int32_t* __restrict__ src, int32_t nsrc, int32_t n,
                                   const int32_t* __restrict__ rp, const int32_t* __restrict__ ci,
                                   const int32_t* __restrict__ dist, const int32_t* __restrict__ dist2,
                                   const int32_t* __restrict__ dist3, unsigned long long* __restrict__ keys) {
    const int lane = threadIdx.x & 31;
    const int warp = (blockIdx.x * blockDim.x + threadIdx.x) >> 5;
    const int nwarp = (gridDim.x * blockDim.x) >> 5;
    auto clamp8 = [](int d) -> unsigned long long { return d < 0 || d > 255 ? 255ull : (unsigned long long)d; };
    for (int i = warp; i < nsrc; i += nwarp) {
        const int s = src != nullptr ? src[i] : i;  // no list: the keys of vertices 0 .. nsrc-1
        if (s < 0 || s >= n) {  // not a vertex: an asynchronous call's check reports it; read nothing
            if (lane == 0) keys[i] = ~0ull;
            continue;
        }
        const int ds = dist[s];
        int best = INT_MAX;
        if (ds > 0)
            for (int e = rp[s] + lane; e < rp[s + 1]; e += 32) {
                int u = ci[e];
                if (dist[u] == ds - 1) best = min(best, u);
            }
        best = warp_min_i32(best);
        if (lane == 0) {
            unsigned long long k = clamp8(ds) << 56;
            if (dist2) k |= clamp8(dist2[s]) << 48 | clamp8(dist3[s]) << 40;
            keys[i] = k | (unsigned)(best == INT_MAX ? s : best);
        }
    }
}

// The vertex of largest degree (smallest id among equals) other than a and b.
__global__ void landmark_kernel(const int32_t* __restrict__ rp, int32_t n, int32_t a, int32_t b,
                                unsigned long long* __restrict__ out) {
    unsigned long long best = 0;
    for (int v = blockIdx.x * blockDim.x + threadIdx.x; v < n; v += gridDim.x * blockDim.x) {
        if (v == a || v == b) continue;
        const unsigned long long key = ((unsigned long long)(unsigned)(rp[v + 1] - rp[v]) << 32) | (unsigned)~(unsigned)v;
        best = key > best ? key : best;
    }
    for (int o = 16; o > 0; o >>= 1) {
        const unsigned long long y = shfl_u64(kFull, best, lane_id() ^ o);
        best = y > best ? y : best;
    }
    if (lane_id() == 0) atomicMax(out, best);
}

// A copy of the call's sources in key order (stable), or nullptr to keep the
// caller's order (a single source, or the plain form).
static int plain_bottom_up(const Graph* g, int32_t opt);

// Hop distances from a maximum-degree vertex (one plain-form BFS per graph,
// kept with the graph): they key the source regrouping, and their largest
// value estimates the diameter, which sizes the plain form's block groups.
static sp_status ensure_top_bfs(Graph* g, cudaStream_t st) {
    std::lock_guard<std::mutex> lk(g->mu);
    if (g->d_top_dist || g->n == 0) return SP_OK;
    int32_t* d_dist = nullptr;
    int32_t* d_one = nullptr;
    SP_CUDA(cudaMalloc((void**)&d_dist, sizeof(int32_t) * (size_t)g->n));
    SP_CUDA(cudaMallocAsync((void**)&d_one, sizeof(int32_t), st));
    SP_CUDA(cudaMemcpyAsync(d_one, &g->top_vertex, sizeof(int32_t), cudaMemcpyHostToDevice, st));
    PlainLaunch L{};
    L.g = g;
    L.d_sources = d_one;
    L.nsrc = 1;
    L.d_dist = d_dist;
    L.mode = PlainMode::BFS;
    L.timeout_ns = bfs_timeout_ns();
    L.stream = st;
    L.bottom_up_den = plain_bottom_up(g, 0);
    LaunchResult r;
    sp_status rc = run_plain(L, &r);
    cudaFreeAsync(d_one, st);
    if (rc == SP_OK) rc = map_device_error(r.err, "eccentricity BFS", r.diag);
    if (rc != SP_OK) {
        cudaFree(d_dist);
        return rc;
    }
    g->d_top_dist = d_dist;
    g->top_levels = r.levels;
    return SP_OK;
}

// Distances from the second and third landmarks (plain-form BFS, kept with
// the graph; computed on the first batched call that regroups sources).
static sp_status ensure_landmarks(Graph* g, cudaStream_t st) {
    std::lock_guard<std::mutex> lk(g->mu);
    if (g->d_land_dist || g->n < 3) return SP_OK;
    unsigned long long* d_key = nullptr;
    int32_t* d_two = nullptr;
    int32_t* d_dist = nullptr;
    SP_CUDA(cudaMallocAsync((void**)&d_key, sizeof(unsigned long long), st));
    int32_t land[2] = {0, 0};
    const int grid = device_sm_count(g->device) * 4;
    for (int k = 0; k < 2; ++k) {
        SP_CUDA(cudaMemsetAsync(d_key, 0, sizeof(unsigned long long), st));
        landmark_kernel<<<grid, 256, 0, st>>>(g->d_rp, g->n, g->top_vertex, k == 0 ? g->top_vertex : land[0], d_key);
        unsigned long long h = 0;
        SP_CUDA(cudaMemcpyAsync(&h, d_key, sizeof(h), cudaMemcpyDeviceToHost, st));
        SP_CUDA(cudaStreamSynchronize(st));
        land[k] = (int32_t)~(unsigned)(h & 0xFFFFFFFFull);
    }
    cudaFreeAsync(d_key, st);
    SP_CUDA(cudaMalloc((void**)&d_dist, sizeof(int32_t) * 2 * (size_t)g->n));
    SP_CUDA(cudaMallocAsync((void**)&d_two, sizeof(int32_t) * 2, st));
    SP_CUDA(cudaMemcpyAsync(d_two, land, sizeof(land), cudaMemcpyHostToDevice, st));
    PlainLaunch L{};
    L.g = g;
    L.d_sources = d_two;
    L.nsrc = 2;
    L.d_dist = d_dist;
    L.mode = PlainMode::BFS;
    L.timeout_ns = bfs_timeout_ns();
    L.stream = st;
    L.bottom_up_den = plain_bottom_up(g, 0);
    LaunchResult r;
    sp_status rc = run_plain(L, &r);
    cudaFreeAsync(d_two, st);
    if (rc == SP_OK) rc = map_device_error(r.err, "landmark BFS", r.diag);
    if (rc != SP_OK) {
        cudaFree(d_dist);
        return rc;
    }
    g->d_land_dist = d_dist;
    return SP_OK;
}

// Blocks per group of the plain form: about 8,192 arcs of an average level
// per block, from the estimated number of levels.
static int plain_group_blocks(const Graph* g) {
    const int64_t levels = std::max<int64_t>(1, g->top_levels);
    const int64_t per_level = std::max<int64_t>(1, g->knnz() / levels);
    return (int)std::min<int64_t>((per_level + 8191) / 8192, 1 << 20);
}

// Bottom-up discovery threshold of the batched form without a trial: the
// caller's, else n/100 on graphs of 750,000 or more vertices (RMAT scale 22,
// width 128: 328 -> 291 ms per launch; ER n = 10^6 / 2·10^6: -9% / -16%;
// RMAT scale 19: +7%), else never.
static int batched_bottom_up(const Graph* g, int32_t opt) {
    if (opt < 0) return 0;
    if (opt > 0) return opt;
    return g->n >= 750000 ? 100 : 0;
}

// Bottom-up discovery threshold of the plain form without a trial: levels
// holding more than n/100 vertices of graphs with at least 2^20 vertices
// (on small graphs the per-lane row scans cost more than the atomics they save).
static int plain_bottom_up(const Graph* g, int32_t opt) {
    if (opt < 0) return 0;
    if (opt > 0) return opt;
    return g->n >= (1 << 20) ? 100 : 0;
}

// Stable sort of the sources by key on the device: a bitonic network over
// (key, position) pairs, ties resolved by position so that equal keys keep
// the caller's order; in one block's shared memory for up to kSortBlockMax
// sources, else in global memory with one launch per merge step.
constexpr int kSortBlockMax = 4096;

__device__ __forceinline__ bool pair_less(unsigned long long ka, unsigned ia, unsigned long long kb, unsigned ib) {
    return ka < kb || (ka == kb && ia < ib);
}

__global__ void sort_sources_block_kernel(const unsigned long long* __restrict__ keys,
                                          const int32_t* __restrict__ src, int32_t m, int32_t p2,
                                          int32_t* __restrict__ out) {
    __shared__ unsigned long long sk[kSortBlockMax];
    __shared__ unsigned si[kSortBlockMax];
    for (int i = threadIdx.x; i < p2; i += blockDim.x) {
        sk[i] = i < m ? keys[i] : ~0ull;
        si[i] = (unsigned)i;
    }
    __syncthreads();
    for (int k = 2; k <= p2; k <<= 1)
        for (int j = k >> 1; j > 0; j >>= 1) {
            for (int i = threadIdx.x; i < p2; i += blockDim.x) {
                const int l = i ^ j;
                if (l > i) {
                    const bool up = (i & k) == 0;
                    const bool gt = pair_less(sk[l], si[l], sk[i], si[i]);
                    if (gt == up) {
                        const unsigned long long tk = sk[i]; sk[i] = sk[l]; sk[l] = tk;
                        const unsigned ti = si[i]; si[i] = si[l]; si[l] = ti;
                    }
                }
            }
            __syncthreads();
        }
    for (int i = threadIdx.x; i < m; i += blockDim.x) out[i] = src[si[i]];
}

__global__ void sort_init_kernel(const unsigned long long* __restrict__ keys, int32_t m, int32_t p2,
                                 unsigned long long* __restrict__ K, unsigned* __restrict__ I) {
    for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < p2; i += gridDim.x * blockDim.x) {
        K[i] = i < m ? keys[i] : ~0ull;
        I[i] = (unsigned)i;
    }
}

__global__ void sort_step_kernel(unsigned long long* __restrict__ K, unsigned* __restrict__ I, int32_t p2, int j,
                                 int k) {
    for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < p2; i += gridDim.x * blockDim.x) {
        const int l = i ^ j;
        if (l <= i) continue;
        const bool up = (i & k) == 0;
        if (pair_less(K[l], I[l], K[i], I[i]) == up) {
            const unsigned long long tk = K[i]; K[i] = K[l]; K[l] = tk;
            const unsigned ti = I[i]; I[i] = I[l]; I[l] = ti;
        }
    }
}

__global__ void sort_gather_kernel(const int32_t* __restrict__ src, const unsigned* __restrict__ I, int32_t m,
                                   int32_t* __restrict__ out) {
    for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < m; i += gridDim.x * blockDim.x) out[i] = src[I[i]];
}

// A copy of the call's sources in key order (stable), built on the device
// without waiting for it; nullptr for fewer than two sources.
static sp_status order_sources(Graph* g, const int32_t* d_src, int32_t nsrc, cudaStream_t st, int32_t** out,
                               int* launches) {
    *out = nullptr;
    if (nsrc < 2 || g->n == 0) return SP_OK;
    {
        sp_status rc = ensure_top_bfs(g, st);
        if (rc != SP_OK) return rc;
    }
    {
        sp_status rc = ensure_landmarks(g, st);
        if (rc != SP_OK) return rc;
    }
    const int32_t* d2 = g->d_land_dist;
    const int32_t* d3 = d2 ? d2 + g->n : nullptr;
    int32_t p2 = 1;
    while (p2 < nsrc) p2 <<= 1;
    const bool one_block = p2 <= kSortBlockMax;
    // keys [nsrc] (+ K [p2], I [p2] for the multi-launch sort) and the output
    const size_t kbytes = sizeof(unsigned long long) * (size_t)nsrc;
    const size_t sbytes = one_block ? 0 : (sizeof(unsigned long long) + sizeof(unsigned)) * (size_t)p2;
    char* buf = nullptr;
    SP_CUDA(cudaMallocAsync((void**)&buf, kbytes + sbytes, st));
    int32_t* sorted = nullptr;
    cudaError_t e = cudaMallocAsync((void**)&sorted, sizeof(int32_t) * (size_t)nsrc, st);
    if (e != cudaSuccess) {
        cudaFreeAsync(buf, st);
        return cuda_fail(e, "source ordering");
    }
    unsigned long long* keys = reinterpret_cast<unsigned long long*>(buf);
    source_keys_kernel<<<std::min(1024, (nsrc + 7) / 8), 256, 0, st>>>(d_src, nsrc, g->n, g->d_rp, g->d_ci,
                                                                          g->d_top_dist, d2, d3, keys);
    int nl = 1;
    if (one_block) {
        sort_sources_block_kernel<<<1, 1024, 0, st>>>(keys, d_src, nsrc, p2, sorted);
        nl += 1;
    } else {
        unsigned long long* K = reinterpret_cast<unsigned long long*>(buf + kbytes);
        unsigned* I = reinterpret_cast<unsigned*>(buf + kbytes + sizeof(unsigned long long) * (size_t)p2);
        const int grid = (int)std::min<int64_t>((p2 + 255) / 256, (int64_t)device_sm_count(g->device) * 8);
        sort_init_kernel<<<grid, 256, 0, st>>>(keys, nsrc, p2, K, I);
        nl += 1;
        for (int k = 2; k <= p2; k <<= 1)
            for (int j = k >> 1; j > 0; j >>= 1) {
                sort_step_kernel<<<grid, 256, 0, st>>>(K, I, p2, j, k);
                nl += 1;
            }
        sort_gather_kernel<<<grid, 256, 0, st>>>(d_src, I, nsrc, sorted);
        nl += 1;
    }
    e = cudaGetLastError();
    cudaFreeAsync(buf, st);
    if (e != cudaSuccess) {
        cudaFreeAsync(sorted, st);
        return cuda_fail(e, "source ordering");
    }
    *out = sorted;
    if (launches) *launches += nl;
    return SP_OK;
}

// Run BC on device buffers, rerunning with a wider representation or more
// workspace when the device reports that it ran out of one.
// d_sq (optional): per vertex, the sum over the sources of delta_s(v)^2
// (the plain and batched forms keep it; a call that asks for it does not run
// the small form).
static sp_status bc_weighted(Graph* g, const int32_t* d_src, int32_t nsrc, const sp_bc_opts& o, double* d_bc,
                             int32_t* d_dist, sp_bc_stats* stats, cudaStream_t st);

static sp_status bc_device(Graph* g, const int32_t* d_src, int32_t nsrc, const sp_bc_opts& o, double* d_bc,
                           sp_bc_stats* stats, cudaStream_t st, double* d_sq) {
    if (g->d_w != nullptr) {
        if (d_sq != nullptr) return fail(SP_ERR_INVALID_ARG, "sampling bounds are not kept for weighted graphs");
        return bc_weighted(g, d_src, nsrc, o, d_bc, nullptr, stats, st);
    }
    absorb_hints(g);
    bool sigma_float;
    {
        std::lock_guard<std::mutex> lk(g->mu);
        sigma_float = g->sigma_float;
    }
    bool theta_f32 = o.precision == SP_FP32_DELTA;
    {
        const int hints = range_hints(g);
        std::lock_guard<std::mutex> lk(g->mu);
        if (hints & 1) g->sigma_float = true;
        if (hints & 2) g->theta_f64 = true;
        if (g->theta_f64) theta_f32 = false;
        sigma_float = g->sigma_float;
    }
    int form = o.form;
    // Automatic form: graphs whose per-source state fits in shared memory run
    // one block per source; otherwise many narrow levels (high diameter)
    // favour small block groups, one source each, and wide levels with many
    // sources favour batches.  Path counts past 64 bits need the plain or
    // batched form's FP64 representation.  Only the latter two need the
    // eccentricity BFS (diameter estimate, group sizes, source regrouping).
    const bool small_fits = (int64_t)g->n <= small_form_max_n(g->device) && d_sq == nullptr;
    if (form == SP_FORM_AUTO && !sigma_float && small_fits) form = SP_FORM_SMALL;
    if (form == SP_FORM_SMALL && !small_fits)
        return fail(SP_ERR_TOO_LARGE, "graph too large for the small form (" + std::to_string(g->n) + " vertices)");
    if (form != SP_FORM_SMALL) {
        sp_status rc = ensure_top_bfs(g, st);
        if (rc != SP_OK) return rc;
    }
    if (form == SP_FORM_AUTO) form = (nsrc >= 2 && g->top_levels <= 64) ? SP_FORM_BATCHED : SP_FORM_PLAIN;
    int width = 1, launches = 0, tuned = 0;
    int batch_bu = batched_bottom_up(g, o.bottom_up);
    if (form == SP_FORM_BATCHED) {
        if (o.batch > 0) {
            width = o.batch;
        } else {
            auto key = tune_key(g, o.precision);
            bool have = false;
            BatchTune t{};
            {
                std::lock_guard<std::mutex> lk(g_tune_mu);
                auto it = g_tuned.find(key);
                if (it != g_tuned.end()) { t = it->second; have = true; }
            }
            if (!have && nsrc >= 128) {
                sp_status trc = autotune_batched(g, d_src, nsrc, o, st, &t, &launches);
                if (trc != SP_OK) return trc;
                tuned = 1;
                // first result wins, so that concurrent calls agree
                std::lock_guard<std::mutex> lk(g_tune_mu);
                t = g_tuned.emplace(key, t).first->second;
                have = true;
            }
            if (have) {
                width = t.width;
                if (o.bottom_up == 0) batch_bu = batched_bottom_up(g, t.bottom_up);
            } else {
                width = default_batch_width(nsrc);
            }
        }
    }
    int driver = 0;
    int bottom_up = o.bottom_up;
    if (form == SP_FORM_PLAIN) {
        driver = o.driver;
        if (o.debug_flags & SP_DEBUG_SKIP_BARRIER) driver = SP_DRIVER_PERSISTENT;
        if (driver == SP_DRIVER_AUTO) {
            auto key = tune_key(g, o.precision);
            bool have = false;
            {
                std::lock_guard<std::mutex> lk(g_tune_mu);
                auto it = g_plain_tune.find(key);
                if (it != g_plain_tune.end() && (o.bottom_up == 0 || it->second.bottom_up == o.bottom_up)) {
                    driver = it->second.driver;
                    bottom_up = it->second.bottom_up;
                    have = true;
                }
            }
            if (!have && nsrc >= 16) {
                PlainTune t{};
                sp_status trc = autotune_plain(g, d_src, o, st, &t, &launches);
                if (trc != SP_OK) return trc;
                tuned = 1;
                std::lock_guard<std::mutex> lk(g_tune_mu);
                if (o.bottom_up == 0) t = g_plain_tune.emplace(key, t).first->second;
                driver = t.driver;
                bottom_up = t.bottom_up;
            }
            if (driver == SP_DRIVER_AUTO) driver = SP_DRIVER_PERSISTENT;
        }
    }
    int32_t* d_sorted = nullptr;
    if (form == SP_FORM_BATCHED && !(o.flags & SP_BC_KEEP_ORDER)) {
        sp_status orc = order_sources(g, d_src, nsrc, st, &d_sorted, &launches);
        if (orc != SP_OK) return orc;
        if (d_sorted) d_src = d_sorted;
    }
    struct FreeSorted {
        int32_t* p;
        cudaStream_t s;
        ~FreeSorted() { if (p) cudaFreeAsync(p, s); }
    } free_sorted{d_sorted, st};
    int promoted = 0, sigma_batches = 0;
    int64_t ecap = 0, hcap = 0, lcap = 0, plain_lcap = 0;
    double kernel_ms = 0.0;
    LaunchResult r;
    for (int attempt = 0; attempt < 16; ++attempt) {
        r = LaunchResult{};
        sp_status rc;
        if (form == SP_FORM_SMALL) {
            SmallLaunch L{};
            L.g = g;
            L.d_sources = d_src;
            L.nsrc = nsrc;
            L.d_bc = d_bc;
            L.theta_f32 = theta_f32;
            L.max_ctas = o.max_ctas;
            L.stream = st;
            rc = run_small(L, &r);
        } else if (form == SP_FORM_PLAIN) {
            PlainLaunch L{};
            L.g = g;
            L.d_sources = d_src;
            L.nsrc = nsrc;
            L.d_bc = d_bc;
            L.mode = PlainMode::BC;
            L.sigma_float = sigma_float;
            L.theta_f32 = theta_f32;
            L.max_ctas = o.max_ctas;
            L.timeout_ns = timeout_of(o);
            L.debug_flags = o.debug_flags;
            L.stream = st;
            L.group_blocks = plain_group_blocks(g);
            L.level_cap = plain_lcap;
            L.bottom_up_den = plain_bottom_up(g, bottom_up);
            L.d_sq = d_sq;
            rc = driver == SP_DRIVER_GRAPH && d_sq == nullptr ? run_plain_graph(L, &r) : run_plain(L, &r);
        } else {
            BatchedLaunch L{};
            L.g = g;
            L.d_sources = d_src;
            L.nsrc = nsrc;
            L.d_bc = d_bc;
            L.width = width;
            L.sigma_float = sigma_float;
            L.theta_f32 = theta_f32;
            L.max_ctas = o.max_ctas;
            L.timeout_ns = timeout_of(o);
            L.debug_flags = o.debug_flags;
            L.stream = st;
            L.entry_cap = ecap;
            L.hub_cap = hcap;
            L.level_cap = lcap;
            L.bottom_up_den = batch_bu;
            L.d_sq = d_sq;
            rc = run_batched(L, &r);
        }
        if (rc != SP_OK) return rc;
        kernel_ms += r.kernel_ms;
        launches += r.launches;
        if (r.err == kErrSigmaOverflow && form == SP_FORM_SMALL) {
            // the small form holds exact counts only: rerun in the plain form
            sp_status trc = ensure_top_bfs(g, st);
            if (trc != SP_OK) return trc;
            form = SP_FORM_PLAIN;
            driver = SP_DRIVER_PERSISTENT;
            sigma_float = true;
            sigma_batches = 1;
            add_range_hint(g, 1);
            std::lock_guard<std::mutex> lk(g->mu);
            g->sigma_float = true;
            continue;
        }
        if (r.err == kErrSigmaOverflow && !sigma_float) {
            sigma_float = true;
            sigma_batches = 1;
            add_range_hint(g, 1);
            std::lock_guard<std::mutex> lk(g->mu);
            g->sigma_float = true;
            continue;
        }
        if (r.err == kErrThetaRange32 && theta_f32) {
            theta_f32 = false;
            promoted = 1;
            add_range_hint(g, 2);
            std::lock_guard<std::mutex> lk(g->mu);
            g->theta_f64 = true;
            continue;
        }
        if (form == SP_FORM_PLAIN && r.err == kErrCapLevels && r.lcap < (int64_t)g->n + 2) {
            plain_lcap = (int64_t)g->n + 2;
            continue;
        }
        if (form == SP_FORM_BATCHED) {
            if (r.err == kErrCapEntries) { ecap = 2 * r.ecap; continue; }
            if (r.err == kErrCapHubs) { hcap = 2 * r.hcap; continue; }
            if (r.err == kErrCapLevels && r.lcap < (int64_t)g->n + 2) { lcap = (int64_t)g->n + 2; continue; }
        }
        break;
    }
    sp_status rc = map_device_error(
        r.err, form == SP_FORM_PLAIN ? "plain form" : (form == SP_FORM_SMALL ? "small form" : "batched form"), r.diag);
    if (rc != SP_OK) return rc;
    if (stats) {
        std::memset(stats, 0, sizeof(*stats));
        stats->traversed_arcs = (int64_t)r.traversed_arcs;
        stats->reached = (int64_t)r.reached;
        stats->entries = (int64_t)r.entries;
        stats->scanned_arcs = (int64_t)r.scanned_arcs;
        stats->max_levels = r.levels;
        stats->batch = width;
        stats->batches = form == SP_FORM_BATCHED ? (nsrc + width - 1) / width : nsrc;
        stats->form = form;
        stats->promoted = promoted || (o.precision == SP_FP32_DELTA && !theta_f32);
        stats->sigma_float = sigma_float ? 1 : sigma_batches;
        stats->dag_arcs = (int64_t)r.dag_arcs;
        stats->recentred = (int32_t)std::min<unsigned long long>(r.recentred, INT32_MAX);
        stats->kernel_ms = kernel_ms;
        stats->launches = launches;
        stats->tuned = tuned;
        stats->driver = form == SP_FORM_PLAIN ? driver : 0;
        stats->bottom_up = form == SP_FORM_PLAIN ? plain_bottom_up(g, bottom_up)
                                                 : (form == SP_FORM_BATCHED ? batch_bu : 0);
    }
    return SP_OK;
}

// The weighted form: reruns with a larger distance cap when a distance
// passes it (up to 2^30).
static sp_status bc_weighted(Graph* g, const int32_t* d_src, int32_t nsrc, const sp_bc_opts& o, double* d_bc,
                             int32_t* d_dist, sp_bc_stats* stats, cudaStream_t st) {
    LaunchResult r;
    int64_t cap = 1 << 18;
    int launches = 0;
    double kernel_ms = 0.0;
    for (int attempt = 0; attempt < 8; ++attempt) {
        WeightedLaunch L{};
        L.g = g;
        L.d_sources = d_src;
        L.nsrc = nsrc;
        L.d_bc = d_bc;
        L.d_dist = d_dist;
        L.dist_cap = cap;
        L.max_ctas = o.max_ctas;
        L.stream = st;
        r = LaunchResult{};
        sp_status rc = run_weighted(L, &r);
        if (rc != SP_OK) return rc;
        launches += r.launches;
        kernel_ms += r.kernel_ms;
        if (r.err == kErrCapLevels && cap < (int64_t)1 << 30) {
            cap = std::min<int64_t>(cap * 8, (int64_t)1 << 30);
            continue;
        }
        break;
    }
    sp_status rc = map_device_error(r.err, "weighted form", r.diag);
    if (rc != SP_OK) return rc;
    if (stats) {
        std::memset(stats, 0, sizeof(*stats));
        stats->traversed_arcs = (int64_t)r.traversed_arcs;
        stats->reached = (int64_t)r.reached;
        stats->entries = (int64_t)r.entries;
        stats->scanned_arcs = (int64_t)r.scanned_arcs;
        stats->max_levels = r.levels;
        stats->batches = nsrc;
        stats->batch = 1;
        stats->form = SP_FORM_WEIGHTED;
        stats->kernel_ms = kernel_ms;
        stats->launches = launches;
    }
    return SP_OK;
}

// Sum of a request's per-word partial BC vectors, in word order.
__global__ void sum_words_kernel(const double* __restrict__ word_bc, int64_t w0, int nw, int64_t n,
                                 double* __restrict__ out) {
    for (int64_t v = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; v < n; v += (int64_t)gridDim.x * blockDim.x) {
        double s = 0.0;
        for (int k = 0; k < nw; ++k) s += word_bc[(w0 + k) * n + v];
        out[v] = s;
    }
}

bool request_is_batched(Graph* g, int32_t nsrc, const sp_bc_opts& o, cudaStream_t st) {
    if (g->d_w != nullptr) return false;  // weighted graphs: the weighted form, request by request
    if (o.form == SP_FORM_BATCHED) return true;
    if (o.form != SP_FORM_AUTO || nsrc < 2 || o.debug_flags != 0) return false;
    bool sigma_float;
    {
        std::lock_guard<std::mutex> lk(g->mu);
        sigma_float = g->sigma_float;
    }
    if (!sigma_float && (int64_t)g->n <= small_form_max_n(g->device)) return false;
    if (ensure_top_bfs(g, st) != SP_OK) return false;
    return g->top_levels <= 64;
}

// Representation and shape of a request-mode launch on g: path counts exact
// or FP64 and dependencies FP32 or FP64 as the graph's earlier calls found
// necessary; the graph's tuned width, else one by the launch's size (a
// request's result does not depend on it: per-word partial vectors); the
// bottom-up threshold.  Makes sure the regrouping BFS distances exist.
struct RequestShape {
    bool sigma_float = false, theta_f32 = false;
    int width = 0, bottom_up = 0;
};
static sp_status request_shape(Graph* g, const sp_bc_opts& o, int64_t nsrc, cudaStream_t st, RequestShape* out) {
    absorb_hints(g);
    out->theta_f32 = o.precision == SP_FP32_DELTA;
    {
        const int hints = range_hints(g);
        std::lock_guard<std::mutex> lk(g->mu);
        if (hints & 1) g->sigma_float = true;
        if (hints & 2) g->theta_f64 = true;
        if (g->theta_f64) out->theta_f32 = false;
        out->sigma_float = g->sigma_float;
    }
    {
        sp_status rc = ensure_top_bfs(g, st);
        if (rc == SP_OK) rc = ensure_landmarks(g, st);
        if (rc != SP_OK) return rc;
    }
    int width = 0;
    out->bottom_up = batched_bottom_up(g, o.bottom_up);
    {
        std::lock_guard<std::mutex> lk(g_tune_mu);
        auto it = g_tuned.find(tune_key(g, o.precision));
        if (it != g_tuned.end()) {
            width = it->second.width;
            if (o.bottom_up == 0) out->bottom_up = batched_bottom_up(g, it->second.bottom_up);
        }
    }
    if (width == 0) width = nsrc >= 128 ? 128 : default_batch_width((int32_t)std::max<int64_t>(nsrc, 1));
    out->width = width;
    return SP_OK;
}

sp_status bc_requests(Graph* g, RequestPart* parts, int nparts, const sp_bc_opts& o, cudaStream_t st) {
    const int64_t n = g->n;
    int64_t total = 0;
    for (int p = 0; p < nparts; ++p) {
        std::memset(&parts[p].stats, 0, sizeof(sp_bc_stats));
        total += parts[p].nsrc;
    }
    if (n == 0 || total == 0) {
        for (int p = 0; p < nparts; ++p)
            if (n > 0) SP_CUDA(cudaMemsetAsync(parts[p].d_out, 0, sizeof(double) * (size_t)n, st));
        SP_CUDA(cudaStreamSynchronize(st));
        return SP_OK;
    }
    RequestShape shape;
    {
        sp_status rc = request_shape(g, o, total, st, &shape);
        if (rc != SP_OK) return rc;
    }
    bool sigma_float = shape.sigma_float, theta_f32 = shape.theta_f32;
    const int width = shape.width, batch_bu = shape.bottom_up;
    const int W = width / 32;

    // Each request's sources regrouped among themselves (same keys as a
    // single call), then laid out request after request in whole words.
    std::vector<int32_t> all((size_t)total);
    {
        int64_t at = 0;
        for (int p = 0; p < nparts; ++p) {
            std::memcpy(all.data() + at, parts[p].h_sources, sizeof(int32_t) * (size_t)parts[p].nsrc);
            at += parts[p].nsrc;
        }
    }
    std::vector<unsigned long long> keys((size_t)total);
    bool have_keys = false;
    {
        std::lock_guard<std::mutex> lk(g->mu);
        if ((int64_t)g->h_keys.size() == n) {  // the graph's host copy (the server makes one per graph)
            for (int64_t i = 0; i < total; ++i) {
                const int32_t x = all[(size_t)i];
                if (x < 0 || x >= n) return fail(SP_ERR_INVALID_ARG, "request source out of range");
                keys[(size_t)i] = g->h_keys[(size_t)x];
            }
            have_keys = true;
        }
    }
    if (!have_keys) {
        int32_t* d_all = nullptr;
        unsigned long long* d_keys = nullptr;
        SP_CUDA(cudaMallocAsync((void**)&d_all, sizeof(int32_t) * (size_t)total, st));
        SP_CUDA(cudaMallocAsync((void**)&d_keys, sizeof(unsigned long long) * (size_t)total, st));
        SP_CUDA(cudaMemcpyAsync(d_all, all.data(), sizeof(int32_t) * (size_t)total, cudaMemcpyHostToDevice, st));
        {
            sp_status rc = check_sources(d_all, (int32_t)total, g->n, st);
            if (rc != SP_OK) { cudaFreeAsync(d_all, st); cudaFreeAsync(d_keys, st); return rc; }
        }
        const int32_t* d2 = g->d_land_dist;
        source_keys_kernel<<<std::min<int64_t>(1024, (total + 7) / 8), 256, 0, st>>>(
            d_all, (int32_t)total, g->n, g->d_rp, g->d_ci, g->d_top_dist, d2, d2 ? d2 + g->n : nullptr, d_keys);
        cudaError_t e = cudaGetLastError();
        if (e == cudaSuccess)
            e = cudaMemcpyAsync(keys.data(), d_keys, sizeof(unsigned long long) * (size_t)total, cudaMemcpyDeviceToHost,
                                st);
        cudaFreeAsync(d_keys, st);
        cudaFreeAsync(d_all, st);
        if (e == cudaSuccess) e = cudaStreamSynchronize(st);
        if (e != cudaSuccess) return cuda_fail(e, "request source ordering");
    }
    std::vector<int64_t> wfirst(nparts), wcount(nparts);
    int64_t words = 0;
    for (int p = 0; p < nparts; ++p) {
        wfirst[p] = words;
        wcount[p] = (parts[p].nsrc + 31) / 32;
        words += wcount[p];
    }
    const int64_t words_pad = (words + W - 1) / W * W;
    std::vector<int32_t> lanes((size_t)words_pad * 32, -1);
    {
        int64_t at = 0;
        for (int p = 0; p < nparts; ++p) {
            const int m = parts[p].nsrc;
            std::vector<int32_t> idx(m);
            for (int i = 0; i < m; ++i) idx[i] = i;
            std::stable_sort(idx.begin(), idx.end(), [&](int32_t x, int32_t y) { return keys[at + x] < keys[at + y]; });
            for (int i = 0; i < m; ++i) lanes[(size_t)wfirst[p] * 32 + i] = all[at + idx[i]];
            at += m;
        }
    }
    if (words_pad * 32 > INT32_MAX) return fail(SP_ERR_TOO_LARGE, "too many sources in one launch");
    int32_t* d_lanes = nullptr;
    double* d_wbc = nullptr;
    unsigned long long* d_wst = nullptr;
    struct Free {
        std::vector<void*> p;
        cudaStream_t s;
        ~Free() { for (void* x : p) if (x) cudaFreeAsync(x, s); }
    } fr{{}, st};
    SP_CUDA(cudaMallocAsync((void**)&d_lanes, sizeof(int32_t) * lanes.size(), st));
    fr.p.push_back(d_lanes);
    if (cudaMallocAsync((void**)&d_wbc, sizeof(double) * (size_t)words_pad * (size_t)n, st) != cudaSuccess) {
        cudaGetLastError();
        return fail(SP_ERR_OOM, "per-word BC vectors");
    }
    fr.p.push_back(d_wbc);
    SP_CUDA(cudaMallocAsync((void**)&d_wst, sizeof(unsigned long long) * 2 * (size_t)words_pad, st));
    fr.p.push_back(d_wst);
    SP_CUDA(cudaMemcpyAsync(d_lanes, lanes.data(), sizeof(int32_t) * lanes.size(), cudaMemcpyHostToDevice, st));

    int promoted = 0, launches = 2;
    int64_t ecap = 0, hcap = 0, lcap = 0;
    double kernel_ms = 0.0;
    LaunchResult r;
    for (int attempt = 0; attempt < 16; ++attempt) {
        SP_CUDA(cudaMemsetAsync(d_wbc, 0, sizeof(double) * (size_t)words_pad * (size_t)n, st));
        SP_CUDA(cudaMemsetAsync(d_wst, 0, sizeof(unsigned long long) * 2 * (size_t)words_pad, st));
        BatchedLaunch L{};
        L.g = g;
        L.d_sources = d_lanes;
        L.nsrc = (int32_t)(words_pad * 32);
        L.d_bc = nullptr;
        L.width = width;
        L.sigma_float = sigma_float;
        L.theta_f32 = theta_f32;
        L.max_ctas = o.max_ctas;
        L.timeout_ns = timeout_of(o);
        L.stream = st;
        L.entry_cap = ecap;
        L.hub_cap = hcap;
        L.level_cap = lcap;
        L.d_word_bc = d_wbc;
        L.d_word_stats = d_wst;
        L.word_cap = (int32_t)words_pad;
        L.bottom_up_den = batch_bu;
        r = LaunchResult{};
        sp_status rc = run_batched(L, &r);
        if (rc != SP_OK) return rc;
        kernel_ms += r.kernel_ms;
        launches += r.launches;
        if (r.err == kErrSigmaOverflow && !sigma_float) {
            sigma_float = true;
            add_range_hint(g, 1);
            std::lock_guard<std::mutex> lk(g->mu);
            g->sigma_float = true;
            continue;
        }
        if (r.err == kErrThetaRange32 && theta_f32) {
            theta_f32 = false;
            promoted = 1;
            add_range_hint(g, 2);
            std::lock_guard<std::mutex> lk(g->mu);
            g->theta_f64 = true;
            continue;
        }
        if (r.err == kErrCapEntries) { ecap = 2 * r.ecap; continue; }
        if (r.err == kErrCapHubs) { hcap = 2 * r.hcap; continue; }
        if (r.err == kErrCapLevels && r.lcap < n + 2) { lcap = n + 2; continue; }
        break;
    }
    sp_status rc = map_device_error(r.err, "batched form (requests)", r.diag);
    if (rc != SP_OK) return rc;
    std::vector<unsigned long long> wst((size_t)words_pad * 2);
    SP_CUDA(cudaMemcpyAsync(wst.data(), d_wst, sizeof(unsigned long long) * wst.size(), cudaMemcpyDeviceToHost, st));
    const int rgrid = (int)std::min<int64_t>((n + 255) / 256, (int64_t)device_sm_count(g->device) * 8);
    for (int p = 0; p < nparts; ++p) {
        sum_words_kernel<<<std::max(rgrid, 1), 256, 0, st>>>(d_wbc, wfirst[p], (int)wcount[p], n, parts[p].d_out);
        SP_CUDA(cudaGetLastError());
    }
    SP_CUDA(cudaStreamSynchronize(st));
    // traversed and reached pairs per request from its words; the launch's
    // other counts split in proportion to traversed pairs
    const double all_arcs = (double)std::max<unsigned long long>(r.traversed_arcs, 1);
    for (int p = 0; p < nparts; ++p) {
        sp_bc_stats& st_p = parts[p].stats;
        unsigned long long arcs = 0, reached = 0;
        for (int64_t k = wfirst[p]; k < wfirst[p] + wcount[p]; ++k) {
            arcs += wst[2 * k];
            reached += wst[2 * k + 1];
        }
        const double share = (double)arcs / all_arcs;
        st_p.traversed_arcs = (int64_t)arcs;
        st_p.reached = (int64_t)reached;
        st_p.entries = (int64_t)(share * (double)r.entries);
        st_p.scanned_arcs = (int64_t)(share * (double)r.scanned_arcs);
        st_p.dag_arcs = (int64_t)(share * (double)r.dag_arcs);
        st_p.kernel_ms = kernel_ms;
        st_p.max_levels = r.levels;
        st_p.batches = (int32_t)(words_pad / W);
        st_p.batch = width;
        st_p.form = SP_FORM_BATCHED;
        st_p.promoted = promoted || (o.precision == SP_FP32_DELTA && !theta_f32);
        st_p.sigma_float = sigma_float ? 1 : 0;
        st_p.recentred = (int32_t)std::min<unsigned long long>(r.recentred, INT32_MAX);
        st_p.launches = launches + nparts;
    }
    return SP_OK;
}

// ---------------------------------------------------------------------------
// Serving: a batched launch that takes requests between its batches (live
// feed).  The host side of the protocol described with FeedCtl / FeedReq.

sp_status graph_host_keys(Graph* g, cudaStream_t st) {
    {
        std::lock_guard<std::mutex> lk(g->mu);
        if ((int64_t)g->h_keys.size() == g->n) return SP_OK;
    }
    if (g->n == 0) return SP_OK;
    sp_status rc = ensure_top_bfs(g, st);
    if (rc == SP_OK) rc = ensure_landmarks(g, st);
    if (rc != SP_OK) return rc;
    std::vector<unsigned long long> keys((size_t)g->n);
    unsigned long long* d_keys = nullptr;
    SP_CUDA(cudaMallocAsync((void**)&d_keys, sizeof(unsigned long long) * (size_t)g->n, st));
    const int32_t* d2 = g->d_land_dist;
    const int grid = (int)std::min<int64_t>((g->n + 7) / 8, (int64_t)device_sm_count(g->device) * 8);
    source_keys_kernel<<<std::max(grid, 1), 256, 0, st>>>(nullptr, g->n, g->n, g->d_rp, g->d_ci, g->d_top_dist, d2,
                                                          d2 ? d2 + g->n : nullptr, d_keys);
    cudaError_t e = cudaGetLastError();
    if (e == cudaSuccess)
        e = cudaMemcpyAsync(keys.data(), d_keys, sizeof(unsigned long long) * (size_t)g->n, cudaMemcpyDeviceToHost, st);
    cudaFreeAsync(d_keys, st);
    if (e == cudaSuccess) e = cudaStreamSynchronize(st);
    if (e != cudaSuccess) return cuda_fail(e, "source keys of the graph");
    std::lock_guard<std::mutex> lk(g->mu);
    g->h_keys.swap(keys);
    return SP_OK;
}

constexpr int32_t kLiveReqs = 256;                 // request slots of a feed
constexpr int32_t kLiveMaxWords = 256;            // word slots of a feed, at most
constexpr size_t kLiveWordBytes = size_t(1) << 30;  // per-word BC vectors of a feed, at most (soft)

sp_status live_open(Graph* g, const sp_bc_opts& o, int64_t nsrc, LiveFeed* lf, cudaStream_t st) {
    const int64_t n = g->n;
    if (n == 0) return fail(SP_ERR_INVALID_ARG, "live feed on an empty graph");
    {
        sp_status rc = graph_host_keys(g, st);
        if (rc != SP_OK) return rc;
    }
    RequestShape shape;
    {
        sp_status rc = request_shape(g, o, nsrc, st, &shape);
        if (rc != SP_OK) return rc;
    }
    const int width = shape.width, batch_bu = shape.bottom_up;
    const bool sigma_float = shape.sigma_float, theta_f32 = shape.theta_f32;
    // word slots: room for the largest request plus a batch, more while the
    // vectors stay within about 1 GiB
    const int64_t min_words = (int64_t)(1024 / 32) + width / 32;
    const int64_t by_bytes = (int64_t)(kLiveWordBytes / (sizeof(double) * (size_t)n));
    const int32_t word_cap = (int32_t)std::max<int64_t>(min_words, std::min<int64_t>(by_bytes, kLiveMaxWords));
    if (lf->ctl == nullptr) {  // first use: the mapped feed, sized for the largest feed
        void* hp = nullptr;
        const size_t o_req = 64, o_lanes = o_req + sizeof(FeedReq) * (size_t)kLiveReqs;
        const size_t bytes = o_lanes + sizeof(int32_t) * 32 * (size_t)kLiveMaxWords;
        cudaError_t e = cudaHostAlloc(&hp, bytes, cudaHostAllocMapped);
        if (e != cudaSuccess) return cuda_fail(e, "live feed");
        std::memset(hp, 0, bytes);
        void* dp = nullptr;
        e = cudaHostGetDevicePointer(&dp, hp, 0);
        if (e != cudaSuccess) {
            cudaFreeHost(hp);
            return cuda_fail(e, "live feed");
        }
        char* h = static_cast<char*>(hp);
        char* d = static_cast<char*>(dp);
        lf->ctl = reinterpret_cast<FeedCtl*>(h);
        lf->req = reinterpret_cast<FeedReq*>(h + o_req);
        lf->lanes = reinterpret_cast<int32_t*>(h + o_lanes);
        lf->ctl_d = reinterpret_cast<FeedCtl*>(d);
        lf->req_d = reinterpret_cast<FeedReq*>(d + o_req);
        lf->lanes_d = reinterpret_cast<int32_t*>(d + o_lanes);
    }
    if (lf->d_lanes == nullptr) {  // the launch's device copies of lanes and records
        cudaError_t e = cudaMallocAsync((void**)&lf->d_lanes, sizeof(int32_t) * 32 * (size_t)kLiveMaxWords, st);
        if (e == cudaSuccess) e = cudaMallocAsync((void**)&lf->d_req, sizeof(FeedReq) * (size_t)kLiveReqs, st);
        if (e != cudaSuccess) {
            cudaGetLastError();
            return fail(SP_ERR_OOM, "live feed: device copies");
        }
    }
    const size_t wbytes = sizeof(double) * (size_t)word_cap * (size_t)n;
    if (lf->wbc_bytes < wbytes || lf->d_wst == nullptr) {  // zeroed once; launches leave them zero
        if (lf->d_wbc) cudaFreeAsync(lf->d_wbc, st);
        lf->d_wbc = nullptr;
        lf->wbc_bytes = 0;
        if (cudaMallocAsync((void**)&lf->d_wbc, wbytes, st) != cudaSuccess) {
            cudaGetLastError();
            lf->d_wbc = nullptr;
            return fail(SP_ERR_OOM, "live feed: per-word BC vectors");
        }
        cudaError_t e = cudaSuccess;
        if (lf->d_wst == nullptr)
            e = cudaMallocAsync((void**)&lf->d_wst, sizeof(unsigned long long) * 2 * (size_t)kLiveMaxWords, st);
        if (e == cudaSuccess) e = cudaMemsetAsync(lf->d_wbc, 0, wbytes, st);
        if (e == cudaSuccess)
            e = cudaMemsetAsync(lf->d_wst, 0, sizeof(unsigned long long) * 2 * (size_t)kLiveMaxWords, st);
        if (e == cudaSuccess) e = cudaStreamSynchronize(st);
        if (e != cudaSuccess) return cuda_fail(e, "live feed");
        lf->wbc_bytes = wbytes;
    }
    lf->g = g;
    lf->word_cap = word_cap;
    lf->req_cap = kLiveReqs;
    lf->width = width;
    lf->bottom_up = batch_bu;
    lf->sigma_float = sigma_float;
    lf->theta_f32 = theta_f32;
    lf->words = lf->nreq = lf->first_open_word = lf->first_open_req = 0;
    lf->pub_words = lf->pub_nreq = 0;
    lf->ctl->words = 0;
    lf->ctl->nreq = 0;
    lf->ctl->ran_words = 0;
    lf->ctl->closed = 0;
    return SP_OK;
}

int64_t live_append(LiveFeed* lf, const int32_t* h_sources, int32_t nsrc, double* d_out) {
    if (nsrc <= 0 || __atomic_load_n(&lf->ctl->closed, __ATOMIC_ACQUIRE) != 0) return -1;
    const int64_t nw = (nsrc + 31) / 32;
    if (lf->words + nw - lf->first_open_word > lf->word_cap) return -1;  // word slots still in use
    if (lf->nreq + 1 - lf->first_open_req > lf->req_cap) return -1;
    if (lf->words + nw > (int64_t(1) << 25)) return -1;  // lane indices stay within int32
    // the request's sources regrouped among themselves, as bc_requests does
    std::vector<int32_t> idx((size_t)nsrc);
    {
        Graph* g = lf->g;
        std::lock_guard<std::mutex> lk(g->mu);
        if ((int64_t)g->h_keys.size() != g->n) return -1;
        for (int32_t i = 0; i < nsrc; ++i) {
            if (h_sources[i] < 0 || h_sources[i] >= g->n) return -1;
            idx[(size_t)i] = i;
        }
        std::stable_sort(idx.begin(), idx.end(), [&](int32_t x, int32_t y) {
            return g->h_keys[(size_t)h_sources[x]] < g->h_keys[(size_t)h_sources[y]];
        });
    }
    for (int64_t j = 0; j < nw; ++j) {
        int32_t* lane = lf->lanes + (size_t)((lf->words + j) % lf->word_cap) * 32;
        for (int l = 0; l < 32; ++l) {
            const int64_t i = j * 32 + l;
            lane[l] = i < nsrc ? h_sources[idx[(size_t)i]] : -1;
        }
    }
    const int64_t r = lf->nreq;
    FeedReq& fr = lf->req[r % lf->req_cap];
    fr.first_word = (int32_t)lf->words;
    fr.nwords = (int32_t)nw;
    fr.out = d_out;
    fr.traversed = 0;
    fr.reached = 0;
    fr.done = 0;
    lf->nreq += 1;
    lf->words += nw;
    return r;
}

void live_publish(LiveFeed* lf) {
    if (lf->pub_words == lf->words) return;
    __atomic_store_n(&lf->ctl->nreq, (int32_t)lf->nreq, __ATOMIC_RELEASE);
    __atomic_store_n(&lf->ctl->words, (int32_t)lf->words, __ATOMIC_RELEASE);
    lf->pub_words = lf->words;
    lf->pub_nreq = lf->nreq;
}

bool live_done(const LiveFeed* lf, int64_t r) {
    return __atomic_load_n(&lf->req[r % lf->req_cap].done, __ATOMIC_ACQUIRE) != 0;
}

void live_retire(LiveFeed* lf) {
    while (lf->first_open_req < lf->nreq && live_done(lf, lf->first_open_req)) ++lf->first_open_req;
    lf->first_open_word =
        lf->first_open_req < lf->nreq ? lf->req[lf->first_open_req % lf->req_cap].first_word : lf->words;
}

int64_t live_ran_words(const LiveFeed* lf) { return __atomic_load_n(&lf->ctl->ran_words, __ATOMIC_ACQUIRE); }

sp_status live_start(LiveFeed* lf, const sp_bc_opts& o, cudaStream_t st, cudaHostFn_t on_done, void* on_done_arg) {
    if (lf->h_ctl == nullptr) {
        void* hp = nullptr;
        cudaError_t e = cudaHostAlloc(&hp, sizeof(Ctl), cudaHostAllocDefault);
        if (e != cudaSuccess) return cuda_fail(e, "live feed control block");
        lf->h_ctl = static_cast<Ctl*>(hp);
    }
    if (lf->ev == nullptr) {
        cudaError_t e = cudaEventCreateWithFlags(&lf->ev, cudaEventDisableTiming);
        if (e != cudaSuccess) {
            lf->ev = nullptr;
            return cuda_fail(e, "live feed event");
        }
    }
    std::memset(lf->h_ctl, 0, sizeof(Ctl));
    BatchedLaunch L{};
    L.g = lf->g;
    L.d_sources = lf->d_lanes;
    L.nsrc = 0;
    L.d_bc = nullptr;
    L.width = lf->width;
    L.sigma_float = lf->sigma_float;
    L.theta_f32 = lf->theta_f32;
    L.max_ctas = o.max_ctas;
    L.timeout_ns = timeout_of(o);
    L.stream = st;
    L.d_word_bc = lf->d_wbc;
    L.d_word_stats = lf->d_wst;
    L.word_cap = lf->word_cap;
    L.bottom_up_den = lf->bottom_up;
    L.feed = lf->ctl_d;
    L.feed_req = lf->req_d;
    L.feed_lanes = lf->lanes_d;
    L.req_dev = lf->d_req;
    L.req_cap = lf->req_cap;
    L.ctl_out = lf->h_ctl;
    L.done_ev = lf->ev;
    L.on_done = on_done;
    L.on_done_arg = on_done_arg;
    LaunchResult r;
    return run_batched(L, &r);
}

bool live_ended(LiveFeed* lf, LaunchResult* result) {
    const cudaError_t q = cudaEventQuery(lf->ev);
    if (q == cudaErrorNotReady) return false;
    *result = LaunchResult{};
    if (q != cudaSuccess) {  // the launch failed as a CUDA call: report it as an error of the launch
        cudaGetLastError();
        result->err = SP_ERR_CUDA;
        return true;
    }
    const Ctl& h = *lf->h_ctl;
    result->err = h.err;
    result->levels = h.max_levels;
    result->traversed_arcs = h.traversed_arcs;
    result->reached = h.reached;
    result->entries = h.entries;
    result->scanned_arcs = h.scanned_arcs;
    result->dag_arcs = h.dag_arcs;
    result->recentred = h.recentred;
    // what a failed launch learnt about the graph, as bc_requests records it
    if (h.err == kErrSigmaOverflow && !lf->sigma_float) {
        add_range_hint(lf->g, 1);
        std::lock_guard<std::mutex> lk(lf->g->mu);
        lf->g->sigma_float = true;
    }
    if (h.err == kErrThetaRange32 && lf->theta_f32) {
        add_range_hint(lf->g, 2);
        std::lock_guard<std::mutex> lk(lf->g->mu);
        lf->g->theta_f64 = true;
    }
    return true;
}

void live_scrub(LiveFeed* lf, cudaStream_t st) {
    if (lf->d_wbc) cudaMemsetAsync(lf->d_wbc, 0, lf->wbc_bytes, st);
    if (lf->d_wst) cudaMemsetAsync(lf->d_wst, 0, sizeof(unsigned long long) * 2 * (size_t)kLiveMaxWords, st);
    cudaStreamSynchronize(st);
    cudaGetLastError();
}

void live_close(LiveFeed* lf, cudaStream_t st) {
    if (lf->d_wbc) cudaFreeAsync(lf->d_wbc, st);
    if (lf->d_wst) cudaFreeAsync(lf->d_wst, st);
    if (lf->d_lanes) cudaFreeAsync(lf->d_lanes, st);
    if (lf->d_req) cudaFreeAsync(lf->d_req, st);
    cudaStreamSynchronize(st);
    if (lf->ctl) cudaFreeHost(lf->ctl);
    if (lf->h_ctl) cudaFreeHost(lf->h_ctl);
    if (lf->ev) cudaEventDestroy(lf->ev);
    cudaGetLastError();
    *lf = LiveFeed{};
}

// ---------------------------------------------------------------------------
// Asynchronous calls: enqueue on the caller's stream and return.  The host
// never waits: sources in a device array are checked by a kernel whose
// verdict the BC kernels read before touching them; a launch ends with a
// finish step that latches a device error in the graph's mapped flags (the
// next call on the graph, or sp_graph_sync, returns it) or, for a condition
// that a wider representation fixes, opens the gate of a fallback launch of
// the plain form with FP64 counts and dependencies, and records a hint so
// that later calls start in the representation that fits.

__global__ void check_sources_async_kernel(const int32_t* __restrict__ s, int32_t nsrc, int32_t n, int* pre_err) {
    for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < nsrc; i += gridDim.x * blockDim.x)
        if (s[i] < 0 || s[i] >= n) atomicCAS(pre_err, 0, (int)SP_ERR_INVALID_ARG);
}

__global__ void finish_async_kernel(const Ctl* __restrict__ ctl, DevFlags* flags, int* fallback) {
    if (threadIdx.x != 0) return;
    const int e = ld_volatile(&ctl->err);
    if (e == 0) return;
    int hint = 0;
    if (e == kErrSigmaOverflow) hint = kHintSigmaFloat;
    else if (e == kErrThetaRange32) hint = kHintThetaF64;
    else if (e == kErrCapEntries) hint = kHintEntries;
    else if (e == kErrCapHubs) hint = kHintHubs;
    if (hint != 0) atomicOr_system(&flags->hints, hint);
    const bool fixable = hint != 0 || e == kErrCapLevels || e == kErrCapacity;
    if (fixable && fallback != nullptr) {
        *fallback = 1;
        return;
    }
    atomicCAS_system(&flags->err, 0, e);
}

sp_status enqueue_finish(const Ctl* d_ctl, const AsyncHooks& h, cudaStream_t st) {
    finish_async_kernel<<<1, 32, 0, st>>>(d_ctl, h.flags, h.fallback);
    SP_CUDA(cudaGetLastError());
    return SP_OK;
}

// Hints that earlier asynchronous calls' launches recorded (read without a
// CUDA call; a launch still running may add more later).
static void absorb_hints(Graph* g) {
    if (!g->flags_host) return;
    const int h = __atomic_exchange_n(&g->flags_host->hints, 0, __ATOMIC_ACQ_REL);
    if (h == 0) return;
    if (h & kHintSigmaFloat) add_range_hint(g, 1);
    if (h & kHintThetaF64) add_range_hint(g, 2);
    std::lock_guard<std::mutex> lk(g->mu);
    if (h & kHintSigmaFloat) g->sigma_float = true;
    if (h & kHintThetaF64) g->theta_f64 = true;
    if (h & kHintEntries) g->ecap_mult = std::min(2 * g->ecap_mult, 1 << 12);
    if (h & kHintHubs) g->hcap_mult = std::min(2 * g->hcap_mult, 1 << 12);
}

// The error an earlier asynchronous call on g latched, taken (cleared).
static sp_status take_latched(Graph* g) {
    if (!g->flags_host) return SP_OK;
    const int e = __atomic_exchange_n(&g->flags_host->err, 0, __ATOMIC_ACQ_REL);
    if (e == 0) return SP_OK;
    return map_device_error(e, "an earlier asynchronous call on this graph");
}

// Enqueue BC over device buffers without waiting.  src_checked: the sources
// were already validated on the host.  Returns SP_NOT_READY (nothing
// enqueued) when the call needs the host first: an autotuning trial that has
// not run for this graph shape, or the graph-driven plain form; the caller
// then runs it synchronously.
static sp_status bc_enqueue(Graph* g, const int32_t* d_src, bool src_checked, int32_t nsrc, const sp_bc_opts& o,
                            double* d_bc, cudaStream_t st) {
    if (g->d_w != nullptr) return SP_NOT_READY;  // the weighted form runs synchronously
    absorb_hints(g);
    bool sigma_float, theta_f32 = o.precision == SP_FP32_DELTA;
    int ecap_mult, hcap_mult;
    {
        const int hints = range_hints(g);
        std::lock_guard<std::mutex> lk(g->mu);
        if (hints & 1) g->sigma_float = true;
        if (hints & 2) g->theta_f64 = true;
        if (g->theta_f64) theta_f32 = false;
        sigma_float = g->sigma_float;
        ecap_mult = g->ecap_mult;
        hcap_mult = g->hcap_mult;
    }
    int form = o.form;
    const bool small_fits = (int64_t)g->n <= small_form_max_n(g->device);
    if (form == SP_FORM_AUTO && !sigma_float && small_fits) form = SP_FORM_SMALL;
    if (form == SP_FORM_SMALL && !small_fits)
        return fail(SP_ERR_TOO_LARGE, "graph too large for the small form (" + std::to_string(g->n) + " vertices)");
    {
        sp_status rc = ensure_top_bfs(g, st);  // once per graph; sizes the fallback's block groups
        if (rc != SP_OK) return rc;
    }
    if (form == SP_FORM_AUTO) form = (nsrc >= 2 && g->top_levels <= 64) ? SP_FORM_BATCHED : SP_FORM_PLAIN;
    int width = 1, batch_bu = batched_bottom_up(g, o.bottom_up), bottom_up = o.bottom_up;
    if (form == SP_FORM_BATCHED) {
        if (o.batch > 0) {
            width = o.batch;
        } else {
            std::lock_guard<std::mutex> lk(g_tune_mu);
            auto it = g_tuned.find(tune_key(g, o.precision));
            if (it != g_tuned.end()) {
                width = it->second.width;
                if (o.bottom_up == 0) batch_bu = batched_bottom_up(g, it->second.bottom_up);
            } else if (nsrc >= 128) {
                return SP_NOT_READY;  // the width tuner runs first, synchronously
            } else {
                width = default_batch_width(nsrc);
            }
        }
    }
    if (form == SP_FORM_PLAIN) {
        int driver = (o.debug_flags & SP_DEBUG_SKIP_BARRIER) ? SP_DRIVER_PERSISTENT : o.driver;
        if (driver == SP_DRIVER_AUTO) {
            std::lock_guard<std::mutex> lk(g_tune_mu);
            auto it = g_plain_tune.find(tune_key(g, o.precision));
            if (it != g_plain_tune.end() && (o.bottom_up == 0 || it->second.bottom_up == o.bottom_up)) {
                driver = it->second.driver;
                bottom_up = it->second.bottom_up;
            } else if (nsrc >= 16) {
                return SP_NOT_READY;  // the driver tuner runs first, synchronously
            } else {
                driver = SP_DRIVER_PERSISTENT;
            }
        }
        if (driver == SP_DRIVER_GRAPH) return SP_NOT_READY;
    }

    // per-call words: [0] the sources' check, [1] the fallback's gate
    int* words = nullptr;
    SP_CUDA(cudaMallocAsync((void**)&words, 2 * sizeof(int), st));
    struct FreeWords {
        int* p;
        int32_t* q;
        cudaStream_t s;
        ~FreeWords() {
            if (q) cudaFreeAsync(q, s);
            cudaFreeAsync(p, s);
        }
    } fw{words, nullptr, st};
    SP_CUDA(cudaMemsetAsync(words, 0, 2 * sizeof(int), st));
    if (!src_checked) {
        check_sources_async_kernel<<<std::min(1024, (nsrc + 255) / 256), 256, 0, st>>>(d_src, nsrc, g->n, words);
        SP_CUDA(cudaGetLastError());
    }
    // FP64 counts and FP64 dependencies in the plain form admit no wider
    // representation: their errors are latched directly.
    const bool widest = form == SP_FORM_PLAIN && sigma_float && !theta_f32;
    AsyncHooks h;
    h.pre_err = src_checked ? nullptr : words;
    h.flags = g->flags_dev;
    h.fallback = widest ? nullptr : words + 1;

    const int32_t* d_run = d_src;
    if (form == SP_FORM_BATCHED && !(o.flags & SP_BC_KEEP_ORDER)) {
        sp_status rc = order_sources(g, d_src, nsrc, st, &fw.q, nullptr);
        if (rc != SP_OK) return rc;
        if (fw.q) d_run = fw.q;
    }
    LaunchResult r;
    sp_status rc;
    if (form == SP_FORM_SMALL) {
        SmallLaunch L{};
        L.g = g;
        L.d_sources = d_run;
        L.nsrc = nsrc;
        L.d_bc = d_bc;
        L.theta_f32 = theta_f32;
        L.max_ctas = o.max_ctas;
        L.stream = st;
        L.async = h;
        rc = run_small(L, &r);
    } else if (form == SP_FORM_PLAIN) {
        PlainLaunch L{};
        L.g = g;
        L.d_sources = d_run;
        L.nsrc = nsrc;
        L.d_bc = d_bc;
        L.mode = PlainMode::BC;
        L.sigma_float = sigma_float;
        L.theta_f32 = theta_f32;
        L.max_ctas = o.max_ctas;
        L.timeout_ns = timeout_of(o);
        L.debug_flags = o.debug_flags;
        L.stream = st;
        L.group_blocks = plain_group_blocks(g);
        L.bottom_up_den = plain_bottom_up(g, bottom_up);
        L.async = h;
        rc = run_plain(L, &r);
    } else {
        BatchedLaunch L{};
        L.g = g;
        L.d_sources = d_run;
        L.nsrc = nsrc;
        L.d_bc = d_bc;
        L.width = width;
        L.sigma_float = sigma_float;
        L.theta_f32 = theta_f32;
        L.max_ctas = o.max_ctas;
        L.timeout_ns = timeout_of(o);
        L.debug_flags = o.debug_flags;
        L.stream = st;
        if (ecap_mult > 1) L.entry_cap = std::max<int64_t>(8 * (int64_t)g->n, 1 << 16) * ecap_mult;
        if (hcap_mult > 1) L.hub_cap = ((g->knnz() / 64) * 4 + 1024) * hcap_mult;
        L.bottom_up_den = batch_bu;
        L.async = h;
        rc = run_batched(L, &r);
    }
    if (rc != SP_OK) return rc;
    if (widest) return SP_OK;
    // The fallback: the plain form with FP64 counts and dependencies, in the
    // caller's source order; its kernels return at once unless the finish
    // step of the launch above opened the gate.
    PlainLaunch F{};
    F.g = g;
    F.d_sources = d_src;
    F.nsrc = nsrc;
    F.d_bc = d_bc;
    F.mode = PlainMode::BC;
    F.sigma_float = true;
    F.theta_f32 = false;
    F.max_ctas = o.max_ctas;
    F.timeout_ns = timeout_of(o);
    F.stream = st;
    F.group_blocks = plain_group_blocks(g);
    F.bottom_up_den = plain_bottom_up(g, 0);
    F.async.gate = words + 1;
    F.async.flags = g->flags_dev;
    LaunchResult r2;
    return run_plain(F, &r2);
}

// ---------------------------------------------------------------------------
// Approximate BC by source sampling.  The paper's BC runs "a few iterations"
// of sources (Section 2; Section 5.1, the BC comparison): here the sources are
// drawn uniformly with replacement, s_i = floor(x_i * n / 2^64) with x_i the
// i-th SplitMix64 output of the seed (Steele, Lea and Flood 2014: state
// seed + (i + 1) * 0x9E3779B97F4A7C15, then the published xor-shift-multiply
// finaliser), and the estimate is BC^(v) = (n / k) sum_i delta_{s_i}(v),
// unbiased for BC over all n sources.  The confidence half-width of
// b(v) = BC(v) / ((n - 1)(n - 2)) is the empirical Bernstein bound (Maurer and
// Pontil 2009, Theorem 4, both sides, a union over the n vertices): with
// Y_i = n delta_{s_i}(v) / ((n - 1)(n - 2)) in [0, R], R = n / (n - 1), L =
// ln(4 n / alpha) and V the sample variance of the Y_i,
//     half(v) = sqrt(2 V L / k) + 7 R L / (3 (k - 1)).
// Rounds of sources run until max_v half(v) <= eps (after at least k_min
// sources) or k reaches k_max; each round doubles k at most.

__device__ __forceinline__ unsigned long long splitmix64(unsigned long long seed, unsigned long long i) {
    unsigned long long z = seed + (i + 1ull) * 0x9E3779B97F4A7C15ull;
    z = (z ^ (z >> 30)) * 0xBF58476D1CE4E5B9ull;
    z = (z ^ (z >> 27)) * 0x94D049BB133111EBull;
    return z ^ (z >> 31);
}

__global__ void draw_sources_kernel(unsigned long long seed, long long first, int32_t count, int32_t n,
                                    int32_t* __restrict__ out) {
    for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < count; i += gridDim.x * blockDim.x)
        out[i] = (int32_t)__umul64hi(splitmix64(seed, (unsigned long long)(first + i)), (unsigned long long)n);
}

// acc += round (sums and squared sums); max of the sample variance of delta.
__global__ void approx_accumulate_kernel(const double* __restrict__ rbc, const double* __restrict__ rsq, int64_t n,
                                         double* __restrict__ sum, double* __restrict__ sq, double k,
                                         unsigned long long* __restrict__ max_var_bits) {
    double best = 0.0;
    for (int64_t v = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; v < n; v += (int64_t)gridDim.x * blockDim.x) {
        const double s = sum[v] + rbc[v], q = sq[v] + rsq[v];
        sum[v] = s;
        sq[v] = q;
        const double mean = s / k;
        const double var = k > 1.0 ? fmax(0.0, (q - k * mean * mean) / (k - 1.0)) : 0.0;
        best = fmax(best, var);
    }
    for (int o = 16; o > 0; o >>= 1) best = fmax(best, __shfl_xor_sync(kFull, best, o));
    if ((threadIdx.x & 31) == 0) atomicMax(max_var_bits, (unsigned long long)__double_as_longlong(best));
}

__global__ void approx_scale_kernel(const double* __restrict__ sum, int64_t n, double scale, double* __restrict__ out) {
    for (int64_t v = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; v < n; v += (int64_t)gridDim.x * blockDim.x)
        out[v] = sum[v] * scale;
}

// The half-width of the normalised confidence interval after k sources, from
// the largest sample variance of delta (all vertices share the second term).
static double approx_half_width(double max_var_delta, double k, double n, double alpha) {
    if (k < 2.0 || n < 3.0) return std::numeric_limits<double>::infinity();
    const double c = n / ((n - 1.0) * (n - 2.0));
    const double L = std::log(4.0 * n / alpha);
    const double R = n / (n - 1.0);
    return std::sqrt(2.0 * c * c * max_var_delta * L / k) + 7.0 * R * L / (3.0 * (k - 1.0));
}

sp_status bc_device_entry(Graph* g, const int32_t* d_src, int32_t nsrc, const sp_bc_opts& o, double* d_bc,
                          sp_bc_stats* stats, cudaStream_t st) {
    return bc_device(g, d_src, nsrc, o, d_bc, stats, st);
}

// PageRank into device memory, waiting for the result (serving requests).
sp_status pagerank_device_entry(Graph* g, double damping, double tol, int32_t max_iter, double* d_pr,
                                PrResult* result, cudaStream_t st) {
    if (g->n == 0) return SP_OK;
    PrLaunch L{};
    L.g = g;
    L.damping = damping;
    L.tol = tol;
    L.max_iter = max_iter;
    L.timeout_ns = bfs_timeout_ns();
    L.stream = st;
    L.d_pr = d_pr;
    sp_status rc = run_pagerank(L, result);
    if (rc == SP_OK) rc = map_device_error(result->err, "pagerank", result->diag);
    cudaError_t e = cudaStreamSynchronize(st);
    if (rc == SP_OK && e != cudaSuccess) rc = cuda_fail(e, "pagerank request");
    return rc;
}

// The graph's mapped flags (error and hint words of asynchronous calls).
static sp_status alloc_flags(Graph* g) {
    void* hp = nullptr;
    cudaError_t e = cudaHostAlloc(&hp, sizeof(DevFlags), cudaHostAllocMapped);
    if (e != cudaSuccess) return cuda_fail(e, "graph flags");
    std::memset(hp, 0, sizeof(DevFlags));
    void* dp = nullptr;
    e = cudaHostGetDevicePointer(&dp, hp, 0);
    if (e != cudaSuccess) {
        cudaFreeHost(hp);
        return cuda_fail(e, "graph flags");
    }
    g->flags_host = static_cast<DevFlags*>(hp);
    g->flags_dev = static_cast<DevFlags*>(dp);
    return SP_OK;
}

}  // namespace sp

using namespace sp;

extern "C" {

const char* sp_status_string(sp_status st) {
    switch (st) {
        case SP_OK: return "SP_OK";
        case SP_NOT_READY: return "SP_NOT_READY";
        case SP_ERR_INVALID_ARG: return "SP_ERR_INVALID_ARG";
        case SP_ERR_OOM: return "SP_ERR_OOM";
        case SP_ERR_CUDA: return "SP_ERR_CUDA";
        case SP_ERR_TOO_LARGE: return "SP_ERR_TOO_LARGE";
        case SP_ERR_RANGE: return "SP_ERR_RANGE";
        case SP_ERR_TIMEOUT: return "SP_ERR_TIMEOUT";
        case SP_ERR_CANCELLED: return "SP_ERR_CANCELLED";
        case SP_ERR_BAD_GRAPH: return "SP_ERR_BAD_GRAPH";
        case SP_ERR_NO_DEVICE: return "SP_ERR_NO_DEVICE";
    }
    return "SP_ERR_UNKNOWN";
}

const char* sp_last_error(void) { return g_last_error.c_str(); }

void sp_bc_opts_default(sp_bc_opts* o) {
    if (!o) return;
    std::memset(o, 0, sizeof(*o));
    o->precision = SP_FP64;
    o->form = SP_FORM_AUTO;
}

sp_status sp_graph_create(const int32_t* row_ptr, const int32_t* col_idx, int32_t n, int64_t nnz, uint32_t flags,
                          sp_stream stream, sp_graph* out) {
    set_last_error("");
    if (!out) return fail(SP_ERR_INVALID_ARG, "out is NULL");
    *out = nullptr;
    if (n < 0 || nnz < 0) return fail(SP_ERR_INVALID_ARG, "negative size");
    if (nnz >= (int64_t)INT32_MAX) return fail(SP_ERR_TOO_LARGE, "nnz must be below 2^31 (int32 row_ptr)");
    if (!row_ptr) return fail(SP_ERR_INVALID_ARG, "row_ptr is NULL");
    if (nnz > 0 && !col_idx) return fail(SP_ERR_INVALID_ARG, "col_idx is NULL");
    if (flags & ~(uint32_t)(SP_GRAPH_CHECK_SYMMETRIC | SP_GRAPH_SORT_ROWS | SP_GRAPH_DIRECTED))
        return fail(SP_ERR_INVALID_ARG, "unknown flag");
    if ((flags & SP_GRAPH_DIRECTED) && (flags & SP_GRAPH_CHECK_SYMMETRIC))
        return fail(SP_ERR_INVALID_ARG, "SP_GRAPH_CHECK_SYMMETRIC does not apply to a directed graph");
    if ((flags & SP_GRAPH_DIRECTED) && 2 * nnz >= (int64_t)INT32_MAX)
        return fail(SP_ERR_TOO_LARGE, "a directed graph needs 2 nnz below 2^31 (out- and in-arc rows)");
    sp_status rc = check_device();
    if (rc == SP_OK) rc = refuse_other_device({row_ptr, col_idx}, "sp_graph_create");
    if (rc != SP_OK) return rc;
    cudaStream_t st = reinterpret_cast<cudaStream_t>(stream);
    Graph* g = new Graph();
    cudaGetDevice(&g->device);
    g->n = n;
    g->nnz = nnz;
    auto cleanup = [&](sp_status s) {
        cudaStreamSynchronize(st);
        if (g->d_rp) cudaFreeAsync(g->d_rp, st);
        if (g->d_ci) cudaFreeAsync(g->d_ci, st);
        if (g->d_crp) cudaFree(g->d_crp);
        if (g->d_cci) cudaFree(g->d_cci);
        if (g->d_odeg) cudaFree(g->d_odeg);
        cudaStreamSynchronize(st);
        delete g;
        return s;
    };
    // the CSR from the library's memory pool: creating a graph after another
    // was destroyed reuses memory that is already mapped
    g->pooled_csr = true;
    if (workspace_alloc((void**)&g->d_rp, sizeof(int32_t) * ((size_t)n + 1), st) != cudaSuccess ||
        workspace_alloc((void**)&g->d_ci, sizeof(int32_t) * (size_t)std::max<int64_t>(nnz, 1), st) != cudaSuccess) {
        cudaGetLastError();
        return cleanup(fail(SP_ERR_OOM, "graph arrays"));
    }
    cudaError_t e = cudaMemcpyAsync(g->d_rp, row_ptr, sizeof(int32_t) * ((size_t)n + 1),
                                    is_device_ptr(row_ptr) ? cudaMemcpyDeviceToDevice : cudaMemcpyHostToDevice, st);
    if (e == cudaSuccess && nnz > 0)
        e = cudaMemcpyAsync(g->d_ci, col_idx, sizeof(int32_t) * (size_t)nnz,
                            is_device_ptr(col_idx) ? cudaMemcpyDeviceToDevice : cudaMemcpyHostToDevice, st);
    if (e != cudaSuccess) return cleanup(cuda_fail(e, "copying the graph"));
    std::string detail;
    if (flags & SP_GRAPH_SORT_ROWS) {
        // row offsets and ids are checked before the sort reads them
        rc = validate_graph(g, 0, st, &detail);
        if (rc == SP_ERR_BAD_GRAPH) return cleanup(fail(rc, detail));
        if (rc != SP_OK) return cleanup(rc);
        rc = sort_rows_device(g->d_rp, g->d_ci, n, nnz, st);
        if (rc != SP_OK) return cleanup(rc);
    }
    rc = validate_graph(g, flags & SP_GRAPH_CHECK_SYMMETRIC, st, &detail);
    if (rc == SP_ERR_BAD_GRAPH) return cleanup(fail(rc, detail));
    if (rc == SP_OK && (flags & SP_GRAPH_DIRECTED)) {
        rc = combined_rows(g->d_rp, g->d_ci, n, nnz, st, &g->d_crp, &g->d_cci, &g->d_odeg);
        g->directed = rc == SP_OK;
    }
    if (rc == SP_OK) rc = alloc_flags(g);
    if (rc != SP_OK) return cleanup(rc);
    g->info.directed = g->directed ? 1 : 0;
    *out = reinterpret_cast<sp_graph>(g);
    return SP_OK;
}

sp_status sp_graph_from_edges(const int32_t* src, const int32_t* dst, int64_t m, int32_t n, uint32_t flags,
                              sp_stream stream, sp_graph* out) {
    set_last_error("");
    if (!out) return fail(SP_ERR_INVALID_ARG, "out is NULL");
    *out = nullptr;
    if (n < 0 || m < 0) return fail(SP_ERR_INVALID_ARG, "negative size");
    if (m > 0 && (!src || !dst)) return fail(SP_ERR_INVALID_ARG, "edge arrays are NULL");
    if (2 * m >= (int64_t)INT32_MAX) return fail(SP_ERR_TOO_LARGE, "2 m must be below 2^31 (int32 row_ptr)");
    if (flags & ~(uint32_t)(SP_GRAPH_CHECK_SYMMETRIC | SP_GRAPH_DIRECTED)) return fail(SP_ERR_INVALID_ARG, "unknown flag");
    if ((flags & SP_GRAPH_DIRECTED) && (flags & SP_GRAPH_CHECK_SYMMETRIC))
        return fail(SP_ERR_INVALID_ARG, "SP_GRAPH_CHECK_SYMMETRIC does not apply to a directed graph");
    const bool directed = (flags & SP_GRAPH_DIRECTED) != 0;
    sp_status rc = check_device();
    if (rc == SP_OK) rc = refuse_other_device({src, dst}, "sp_graph_from_edges");
    if (rc != SP_OK) return rc;
    cudaStream_t st = reinterpret_cast<cudaStream_t>(stream);
    int32_t* d_src = nullptr;
    int32_t* d_dst = nullptr;
    auto stage = [&](const int32_t* p, int32_t** d) -> sp_status {
        if (m == 0) return SP_OK;
        if (is_device_ptr(p)) { *d = const_cast<int32_t*>(p); return SP_OK; }
        SP_CUDA(cudaMallocAsync((void**)d, sizeof(int32_t) * (size_t)m, st));
        SP_CUDA(cudaMemcpyAsync(*d, p, sizeof(int32_t) * (size_t)m, cudaMemcpyHostToDevice, st));
        return SP_OK;
    };
    struct Free {
        const int32_t *hs, *hd;
        int32_t *ds, *dd;
        cudaStream_t s;
        ~Free() {
            if (ds && ds != hs) cudaFreeAsync(ds, s);
            if (dd && dd != hd) cudaFreeAsync(dd, s);
        }
    };
    rc = stage(src, &d_src);
    if (rc == SP_OK) rc = stage(dst, &d_dst);
    Free fr{src, dst, d_src, d_dst, st};
    if (rc != SP_OK) return rc;
    Graph* g = new Graph();
    cudaGetDevice(&g->device);
    g->n = n;
    std::string detail;
    rc = csr_from_edges(d_src, d_dst, m, n, directed, st, &g->d_rp, &g->d_ci, &g->nnz, &detail);
    if (rc == SP_OK) rc = validate_graph(g, flags & SP_GRAPH_CHECK_SYMMETRIC, st, &detail);
    if (rc == SP_OK && directed) {
        rc = combined_rows(g->d_rp, g->d_ci, n, g->nnz, st, &g->d_crp, &g->d_cci, &g->d_odeg);
        g->directed = rc == SP_OK;
    }
    if (rc == SP_OK) rc = alloc_flags(g);
    if (rc != SP_OK) {
        if (g->d_rp) cudaFree(g->d_rp);
        if (g->d_ci) cudaFree(g->d_ci);
        if (g->d_crp) cudaFree(g->d_crp);
        if (g->d_cci) cudaFree(g->d_cci);
        if (g->d_odeg) cudaFree(g->d_odeg);
        delete g;
        return rc == SP_ERR_BAD_GRAPH ? fail(rc, detail) : rc;
    }
    g->info.directed = g->directed ? 1 : 0;
    *out = reinterpret_cast<sp_graph>(g);
    return SP_OK;
}

sp_status sp_graph_get_csr(sp_graph gh, int32_t* row_ptr_out, int32_t* col_idx_out, sp_stream stream) {
    set_last_error("");
    if (!gh || !row_ptr_out || !col_idx_out) return fail(SP_ERR_INVALID_ARG, "NULL argument");
    Graph* g = reinterpret_cast<Graph*>(gh);
    {
        sp_status rc = refuse_other_device({row_ptr_out, col_idx_out}, "sp_graph_get_csr");
        if (rc != SP_OK) return rc;
    }
    cudaStream_t st = reinterpret_cast<cudaStream_t>(stream);
    auto kind = [](const void* p) { return is_device_ptr(p) ? cudaMemcpyDeviceToDevice : cudaMemcpyDeviceToHost; };
    cudaError_t e = cudaMemcpyAsync(row_ptr_out, g->d_rp, sizeof(int32_t) * ((size_t)g->n + 1), kind(row_ptr_out), st);
    if (e == cudaSuccess && g->nnz > 0)
        e = cudaMemcpyAsync(col_idx_out, g->d_ci, sizeof(int32_t) * (size_t)g->nnz, kind(col_idx_out), st);
    if (e == cudaSuccess) e = cudaStreamSynchronize(st);
    if (e != cudaSuccess) return cuda_fail(e, "copying the CSR");
    return SP_OK;
}

sp_status sp_graph_destroy(sp_graph gh) {
    if (!gh) return fail(SP_ERR_INVALID_ARG, "graph is NULL");
    Graph* g = reinterpret_cast<Graph*>(gh);
    if (g->d_top_dist) cudaFree(g->d_top_dist);
    if (g->d_land_dist) cudaFree(g->d_land_dist);
    destroy_step_cache(g);
    destroy_pr_plan(g);
    cudaDeviceSynchronize();  // waits for work still running on the graph
    if (g->pooled_csr) {
        cudaFreeAsync(g->d_rp, 0);
        cudaFreeAsync(g->d_ci, 0);
        cudaStreamSynchronize(0);
    } else {
        cudaFree(g->d_rp);
        cudaFree(g->d_ci);
    }
    if (g->d_crp) cudaFree(g->d_crp);
    if (g->d_cci) cudaFree(g->d_cci);
    if (g->d_odeg) cudaFree(g->d_odeg);
    if (g->d_w) cudaFree(g->d_w);
    if (g->flags_host) cudaFreeHost(g->flags_host);
    delete g;
    return SP_OK;
}

sp_status sp_graph_set_weights(sp_graph gh, const int32_t* weights, sp_stream stream) {
    set_last_error("");
    if (!gh) return fail(SP_ERR_INVALID_ARG, "graph is NULL");
    Graph* g = reinterpret_cast<Graph*>(gh);
    if (g->nnz > 0 && !weights) return fail(SP_ERR_INVALID_ARG, "weights is NULL");
    {
        sp_status rc = refuse_other_device({weights}, "sp_graph_set_weights");
        if (rc != SP_OK) return rc;
    }
    return set_weights(g, weights, g->nnz > 0 && is_device_ptr(weights), reinterpret_cast<cudaStream_t>(stream));
}

sp_status sp_sssp(sp_graph gh, const int32_t* sources, int32_t nsrc, int32_t* dist_out, sp_stream stream) {
    set_last_error("");
    if (!gh) return fail(SP_ERR_INVALID_ARG, "graph is NULL");
    Graph* g = reinterpret_cast<Graph*>(gh);
    if (!g->d_w) return fail(SP_ERR_INVALID_ARG, "the graph has no weights (sp_graph_set_weights)");
    if (nsrc < 0) return fail(SP_ERR_INVALID_ARG, "nsrc < 0");
    if (nsrc == 0 || g->n == 0) return SP_OK;
    if (!sources || !dist_out) return fail(SP_ERR_INVALID_ARG, "NULL pointer");
    {
        sp_status rc = take_latched(g);
        if (rc == SP_OK) rc = refuse_other_device({sources, dist_out}, "sp_sssp");
        if (rc != SP_OK) return rc;
    }
    cudaStream_t st = reinterpret_cast<cudaStream_t>(stream);
    const size_t count = (size_t)nsrc * (size_t)g->n;
    const bool host_out = !is_device_ptr(dist_out);
    int32_t* d_dist = dist_out;
    if (host_out) SP_CUDA(cudaMallocAsync((void**)&d_dist, sizeof(int32_t) * count, st));
    int32_t* d_src = nullptr;
    sp_status rc = stage_in(sources, nsrc, st, &d_src);
    if (rc == SP_OK) rc = check_sources(d_src, nsrc, g->n, st);
    sp_bc_opts o;
    sp_bc_opts_default(&o);
    if (rc == SP_OK) rc = bc_weighted(g, d_src, nsrc, o, nullptr, d_dist, nullptr, st);
    if (rc == SP_OK && host_out) {
        cudaError_t e = cudaMemcpyAsync(dist_out, d_dist, sizeof(int32_t) * count, cudaMemcpyDeviceToHost, st);
        if (e != cudaSuccess) rc = cuda_fail(e, "copying dist_out");
    }
    if (d_src) cudaFreeAsync(d_src, st);
    if (host_out) cudaFreeAsync(d_dist, st);
    cudaError_t e = cudaStreamSynchronize(st);
    if (rc == SP_OK && e != cudaSuccess) rc = cuda_fail(e, "sp_sssp");
    return rc;
}

sp_status sp_graph_sync(sp_graph gh, sp_stream stream) {
    set_last_error("");
    if (!gh) return fail(SP_ERR_INVALID_ARG, "graph is NULL");
    Graph* g = reinterpret_cast<Graph*>(gh);
    cudaError_t e = cudaStreamSynchronize(reinterpret_cast<cudaStream_t>(stream));
    if (e != cudaSuccess) return cuda_fail(e, "sp_graph_sync");
    absorb_hints(g);
    return take_latched(g);
}

sp_status sp_graph_get_info(sp_graph gh, sp_graph_info* out) {
    if (!gh || !out) return fail(SP_ERR_INVALID_ARG, "NULL argument");
    *out = reinterpret_cast<Graph*>(gh)->info;
    return SP_OK;
}

sp_status sp_bc_ex(sp_graph gh, const int32_t* sources, int32_t nsrc, const sp_bc_opts* opts, double* bc_out,
                   sp_bc_stats* stats, sp_stream stream) {
    set_last_error("");
    if (!gh) return fail(SP_ERR_INVALID_ARG, "graph is NULL");
    Graph* g = reinterpret_cast<Graph*>(gh);
    if (nsrc < 0) return fail(SP_ERR_INVALID_ARG, "nsrc < 0");
    if (nsrc > 0 && !sources) return fail(SP_ERR_INVALID_ARG, "sources is NULL");
    if (g->n > 0 && !bc_out) return fail(SP_ERR_INVALID_ARG, "bc_out is NULL");
    sp_bc_opts o;
    sp_bc_opts_default(&o);
    if (opts) o = *opts;
    if (o.precision != SP_FP64 && o.precision != SP_FP32_DELTA) return fail(SP_ERR_INVALID_ARG, "precision");
    if (o.form < SP_FORM_AUTO || o.form > SP_FORM_WEIGHTED) return fail(SP_ERR_INVALID_ARG, "form");
    if ((o.form == SP_FORM_WEIGHTED) != (g->d_w != nullptr) && o.form != SP_FORM_AUTO)
        return fail(SP_ERR_INVALID_ARG, "SP_FORM_WEIGHTED is the form of graphs with weights, and theirs only");
    if (o.batch != 0 && o.batch != 32 && o.batch != 64 && o.batch != 128 && o.batch != 256)
        return fail(SP_ERR_INVALID_ARG, "batch must be 0, 32, 64, 128 or 256");
    if (o.max_ctas < 0 || o.barrier_timeout_ns < 0 || o.bottom_up < -1) return fail(SP_ERR_INVALID_ARG, "negative option");
    if (o.driver < SP_DRIVER_AUTO || o.driver > SP_DRIVER_GRAPH) return fail(SP_ERR_INVALID_ARG, "driver");
    if (o.flags & ~(int32_t)SP_BC_KEEP_ORDER) return fail(SP_ERR_INVALID_ARG, "unknown flag");
    {
        sp_status rc = refuse_other_device({sources, bc_out}, "sp_bc");
        if (rc != SP_OK) return rc;
    }
    cudaStream_t st = reinterpret_cast<cudaStream_t>(stream);
    if (stats) std::memset(stats, 0, sizeof(*stats));
    {
        sp_status rc = take_latched(g);
        if (rc != SP_OK) return rc;
    }
    if (g->n == 0) return SP_OK;
    const bool host_out = !is_device_ptr(bc_out);
    if (!host_out && !stats) {
        // Asynchronous: enqueue on `stream` and return.  Host sources are
        // checked here and staged (the copy reads them before return);
        // device sources are read in place by the kernels.
        const bool dev_src = nsrc > 0 && is_device_ptr(sources);
        int32_t* staged = nullptr;
        if (nsrc > 0 && !dev_src) {
            for (int32_t i = 0; i < nsrc; ++i)
                if (sources[i] < 0 || sources[i] >= g->n)
                    return fail(SP_ERR_INVALID_ARG, "source " + std::to_string(i) + " is not a vertex id in [0, n)");
            sp_status rc = stage_in(sources, nsrc, st, &staged);
            if (rc != SP_OK) return rc;
        }
        sp_status rc;
        if (nsrc == 0) {
            cudaError_t e = cudaMemsetAsync(bc_out, 0, sizeof(double) * (size_t)g->n, st);
            rc = e == cudaSuccess ? SP_OK : cuda_fail(e, "zeroing bc_out");
        } else {
            rc = bc_enqueue(g, dev_src ? sources : staged, !dev_src, nsrc, o, bc_out, st);
        }
        if (staged) cudaFreeAsync(staged, st);
        if (rc != SP_NOT_READY) return rc;
        set_last_error("");  // needs a host decision first: run synchronously below
    }
    double* d_bc = bc_out;
    if (host_out) SP_CUDA(cudaMallocAsync((void**)&d_bc, sizeof(double) * (size_t)g->n, st));
    int32_t* d_src = nullptr;
    sp_status rc = stage_in(sources, nsrc, st, &d_src);
    if (rc == SP_OK) rc = check_sources(d_src, nsrc, g->n, st);
    if (rc == SP_OK) {
        if (nsrc == 0) {
            cudaError_t e = cudaMemsetAsync(d_bc, 0, sizeof(double) * (size_t)g->n, st);
            if (e != cudaSuccess) rc = cuda_fail(e, "zeroing bc_out");
        } else {
            rc = bc_device(g, d_src, nsrc, o, d_bc, stats, st);
            if (stats) stats->launches += 1;  // the source check
        }
    }
    if (rc == SP_OK && host_out) {
        cudaError_t e = cudaMemcpyAsync(bc_out, d_bc, sizeof(double) * (size_t)g->n, cudaMemcpyDeviceToHost, st);
        if (e != cudaSuccess) rc = cuda_fail(e, "copying bc_out");
    }
    if (d_src) cudaFreeAsync(d_src, st);
    if (host_out) cudaFreeAsync(d_bc, st);
    cudaError_t e = cudaStreamSynchronize(st);
    if (rc == SP_OK && e != cudaSuccess) rc = cuda_fail(e, "sp_bc");
    return rc;
}

sp_status sp_bc(sp_graph g, const int32_t* sources, int32_t nsrc, double* bc_out, sp_stream stream) {
    return sp_bc_ex(g, sources, nsrc, nullptr, bc_out, nullptr, stream);
}

sp_status sp_bfs(sp_graph gh, const int32_t* sources, int32_t nsrc, int32_t* dist_out, sp_stream stream) {
    set_last_error("");
    if (!gh) return fail(SP_ERR_INVALID_ARG, "graph is NULL");
    Graph* g = reinterpret_cast<Graph*>(gh);
    if (nsrc < 0) return fail(SP_ERR_INVALID_ARG, "nsrc < 0");
    {
        sp_status rc = take_latched(g);
        if (rc != SP_OK) return rc;
    }
    if (nsrc == 0 || g->n == 0) return SP_OK;
    if (!sources || !dist_out) return fail(SP_ERR_INVALID_ARG, "NULL pointer");
    {
        sp_status rc = refuse_other_device({sources, dist_out}, "sp_bfs");
        if (rc != SP_OK) return rc;
    }
    cudaStream_t st = reinterpret_cast<cudaStream_t>(stream);
    const size_t count = (size_t)nsrc * (size_t)g->n;
    const bool host_out = !is_device_ptr(dist_out);
    int32_t* d_dist = dist_out;
    if (host_out) SP_CUDA(cudaMallocAsync((void**)&d_dist, sizeof(int32_t) * count, st));
    int32_t* d_src = nullptr;
    sp_status rc = stage_in(sources, nsrc, st, &d_src);
    if (rc == SP_OK) rc = check_sources(d_src, nsrc, g->n, st);
    if (rc == SP_OK) {
        PlainLaunch L{};
        L.g = g;
        L.d_sources = d_src;
        L.nsrc = nsrc;
        L.d_dist = d_dist;
        L.mode = PlainMode::BFS;
        L.sigma_float = false;
        L.theta_f32 = false;
        L.timeout_ns = bfs_timeout_ns();
        L.stream = st;
        rc = ensure_top_bfs(g, st);
        L.group_blocks = plain_group_blocks(g);
        L.bottom_up_den = plain_bottom_up(g, 0);
        LaunchResult r;
        for (int attempt = 0; rc == SP_OK && attempt < 2; ++attempt) {
            rc = run_plain(L, &r);
            if (rc == SP_OK && r.err == kErrCapLevels && L.level_cap < (int64_t)g->n + 2) {
                L.level_cap = (int64_t)g->n + 2;
                continue;
            }
            break;
        }
        if (rc == SP_OK) rc = map_device_error(r.err, "bfs", r.diag);
    }
    if (rc == SP_OK && host_out) {
        cudaError_t e = cudaMemcpyAsync(dist_out, d_dist, sizeof(int32_t) * count, cudaMemcpyDeviceToHost, st);
        if (e != cudaSuccess) rc = cuda_fail(e, "copying dist_out");
    }
    if (d_src) cudaFreeAsync(d_src, st);
    if (host_out) cudaFreeAsync(d_dist, st);
    cudaError_t e = cudaStreamSynchronize(st);
    if (rc == SP_OK && e != cudaSuccess) rc = cuda_fail(e, "sp_bfs");
    return rc;
}

sp_status sp_bc_approx(sp_graph gh, uint64_t seed, double eps, double alpha, int64_t k_min, int64_t k_max,
                       const sp_bc_opts* opts, double* bc_out, sp_approx_stats* stats, sp_stream stream) {
    set_last_error("");
    if (!gh) return fail(SP_ERR_INVALID_ARG, "graph is NULL");
    Graph* g = reinterpret_cast<Graph*>(gh);
    if (!(eps > 0.0) || !(alpha > 0.0 && alpha < 1.0)) return fail(SP_ERR_INVALID_ARG, "eps > 0 and 0 < alpha < 1");
    if (k_min < 2 || k_max < k_min || k_max > INT32_MAX) return fail(SP_ERR_INVALID_ARG, "2 <= k_min <= k_max < 2^31");
    if (g->n > 0 && !bc_out) return fail(SP_ERR_INVALID_ARG, "bc_out is NULL");
    sp_bc_opts o;
    sp_bc_opts_default(&o);
    if (opts) o = *opts;
    if (o.precision != SP_FP64 && o.precision != SP_FP32_DELTA) return fail(SP_ERR_INVALID_ARG, "precision");
    if (o.form == SP_FORM_SMALL) o.form = SP_FORM_AUTO;  // the small form keeps no squared dependencies
    {
        sp_status rc = take_latched(g);
        if (rc == SP_OK) rc = refuse_other_device({bc_out}, "sp_bc_approx");
        if (rc != SP_OK) return rc;
    }
    if (stats) std::memset(stats, 0, sizeof(*stats));
    if (g->n == 0) return SP_OK;
    cudaStream_t st = reinterpret_cast<cudaStream_t>(stream);
    const int64_t n = g->n;
    {
        sp_status rc = ensure_top_bfs(g, st);
        if (rc != SP_OK) return rc;
    }
    if (o.form == SP_FORM_AUTO) o.form = g->top_levels <= 64 ? SP_FORM_BATCHED : SP_FORM_PLAIN;
    const bool host_out = !is_device_ptr(bc_out);
    // workspace: sum, sq, round bc, round sq [n] each, sources [k_max chunk], max bits
    double *sum = nullptr, *sq = nullptr, *rbc = nullptr, *rsq = nullptr;
    int32_t* src = nullptr;
    unsigned long long* maxv = nullptr;
    struct Free {
        std::vector<void*> p;
        cudaStream_t s;
        ~Free() { for (void* x : p) if (x) cudaFreeAsync(x, s); }
    } fr{{}, st};
    const int64_t chunk_max = std::min<int64_t>(k_max, 1 << 20);
    for (double** p : {&sum, &sq, &rbc, &rsq}) {
        SP_CUDA(cudaMallocAsync((void**)p, sizeof(double) * (size_t)n, st));
        fr.p.push_back(*p);
    }
    SP_CUDA(cudaMallocAsync((void**)&src, sizeof(int32_t) * (size_t)chunk_max, st));
    fr.p.push_back(src);
    SP_CUDA(cudaMallocAsync((void**)&maxv, sizeof(unsigned long long), st));
    fr.p.push_back(maxv);
    SP_CUDA(cudaMemsetAsync(sum, 0, sizeof(double) * (size_t)n, st));
    SP_CUDA(cudaMemsetAsync(sq, 0, sizeof(double) * (size_t)n, st));
    const int egrid = (int)std::min<int64_t>((n + 255) / 256, (int64_t)device_sm_count(g->device) * 8);
    int64_t k = 0;
    int rounds = 0;
    double half = std::numeric_limits<double>::infinity(), kernel_ms = 0.0;
    while (k < k_max) {
        int64_t want = k == 0 ? k_min : std::max<int64_t>(k, 256);  // at most doubles k
        want = std::min(want, std::min(k_max - k, chunk_max));
        draw_sources_kernel<<<(int)std::min<int64_t>((want + 255) / 256, 4096), 256, 0, st>>>(
            (unsigned long long)seed, (long long)k, (int32_t)want, (int32_t)n, src);
        SP_CUDA(cudaGetLastError());
        sp_bc_stats rs{};
        sp_status rc = bc_device(g, src, (int32_t)want, o, rbc, &rs, st, rsq);
        if (rc != SP_OK) return rc;
        kernel_ms += rs.kernel_ms;
        k += want;
        ++rounds;
        SP_CUDA(cudaMemsetAsync(maxv, 0, sizeof(unsigned long long), st));
        approx_accumulate_kernel<<<std::max(egrid, 1), 256, 0, st>>>(rbc, rsq, n, sum, sq, (double)k, maxv);
        SP_CUDA(cudaGetLastError());
        unsigned long long bits = 0;
        SP_CUDA(cudaMemcpyAsync(&bits, maxv, sizeof(bits), cudaMemcpyDeviceToHost, st));
        SP_CUDA(cudaStreamSynchronize(st));
        double max_var;
        std::memcpy(&max_var, &bits, sizeof(max_var));
        half = approx_half_width(max_var, (double)k, (double)n, alpha);
        if (k >= k_min && half <= eps) break;
    }
    double* d_out = bc_out;
    if (host_out) d_out = rbc;  // the round buffer holds the estimate, then it is copied out
    approx_scale_kernel<<<std::max(egrid, 1), 256, 0, st>>>(sum, n, (double)n / (double)k, d_out);
    SP_CUDA(cudaGetLastError());
    if (host_out) SP_CUDA(cudaMemcpyAsync(bc_out, rbc, sizeof(double) * (size_t)n, cudaMemcpyDeviceToHost, st));
    SP_CUDA(cudaStreamSynchronize(st));
    if (stats) {
        stats->sources = k;
        stats->rounds = rounds;
        stats->converged = half <= eps ? 1 : 0;
        stats->bound = half;
        stats->kernel_ms = kernel_ms;
    }
    return SP_OK;
}

sp_status sp_pagerank(sp_graph gh, double damping, double tol, int32_t max_iter, double* pr_out,
                      int32_t* iterations_out, double* change_out, sp_stream stream) {
    set_last_error("");
    if (!gh) return fail(SP_ERR_INVALID_ARG, "graph is NULL");
    Graph* g = reinterpret_cast<Graph*>(gh);
    if (!(damping >= 0.0 && damping <= 1.0)) return fail(SP_ERR_INVALID_ARG, "damping must be in [0, 1]");
    if (max_iter < 0) return fail(SP_ERR_INVALID_ARG, "max_iter < 0");
    if (g->n > 0 && !pr_out) return fail(SP_ERR_INVALID_ARG, "pr_out is NULL");
    {
        sp_status rc = take_latched(g);
        if (rc == SP_OK) rc = refuse_other_device({pr_out}, "sp_pagerank");
        if (rc != SP_OK) return rc;
    }
    if (iterations_out) *iterations_out = 0;
    if (change_out) *change_out = 0.0;
    if (g->n == 0) return SP_OK;
    cudaStream_t st = reinterpret_cast<cudaStream_t>(stream);
    const bool host_out = !is_device_ptr(pr_out);
    PrLaunch L{};
    L.g = g;
    L.damping = damping;
    L.tol = tol;
    L.max_iter = max_iter;
    L.timeout_ns = bfs_timeout_ns();
    L.stream = st;
    PrResult r;
    if (!host_out && !iterations_out && !change_out) {  // asynchronous: nothing to read back
        L.d_pr = pr_out;
        L.async.flags = g->flags_dev;
        return run_pagerank(L, &r);
    }
    double* d_pr = pr_out;
    if (host_out) SP_CUDA(cudaMallocAsync((void**)&d_pr, sizeof(double) * (size_t)g->n, st));
    L.d_pr = d_pr;
    sp_status rc = run_pagerank(L, &r);
    if (rc == SP_OK) rc = map_device_error(r.err, "pagerank", r.diag);
    if (rc == SP_OK && host_out) {
        cudaError_t e = cudaMemcpyAsync(pr_out, d_pr, sizeof(double) * (size_t)g->n, cudaMemcpyDeviceToHost, st);
        if (e != cudaSuccess) rc = cuda_fail(e, "copying pr_out");
    }
    if (host_out) cudaFreeAsync(d_pr, st);
    cudaError_t e = cudaStreamSynchronize(st);
    if (rc == SP_OK && e != cudaSuccess) rc = cuda_fail(e, "sp_pagerank");
    if (rc == SP_OK) {
        if (iterations_out) *iterations_out = r.iterations;
        if (change_out) *change_out = r.change;
    }
    return rc;
}

sp_status sp_sigma(sp_graph gh, int32_t src, double* mant_out, int64_t* exp2_out, sp_stream stream) {
    set_last_error("");
    if (!gh) return fail(SP_ERR_INVALID_ARG, "graph is NULL");
    Graph* g = reinterpret_cast<Graph*>(gh);
    {
        sp_status rc = take_latched(g);
        if (rc != SP_OK) return rc;
    }
    if (src < 0 || src >= g->n) return fail(SP_ERR_INVALID_ARG, "source out of range");
    if (!mant_out || !exp2_out) return fail(SP_ERR_INVALID_ARG, "NULL pointer");
    {
        sp_status rc = refuse_other_device({mant_out, exp2_out}, "sp_sigma");
        if (rc != SP_OK) return rc;
    }
    cudaStream_t st = reinterpret_cast<cudaStream_t>(stream);
    const size_t n = (size_t)g->n;
    const bool host_m = !is_device_ptr(mant_out), host_e = !is_device_ptr(exp2_out);
    double* d_m = mant_out;
    long long* d_e = reinterpret_cast<long long*>(exp2_out);
    if (host_m) SP_CUDA(cudaMallocAsync((void**)&d_m, sizeof(double) * n, st));
    if (host_e) SP_CUDA(cudaMallocAsync((void**)&d_e, sizeof(long long) * n, st));
    int32_t* d_src = nullptr;
    sp_status rc = stage_in(&src, 1, st, &d_src);
    if (rc == SP_OK) {
        PlainLaunch L{};
        L.g = g;
        L.d_sources = d_src;
        L.nsrc = 1;
        L.d_mant = d_m;
        L.d_exp = d_e;
        L.mode = PlainMode::SIGMA;
        L.sigma_float = true;
        L.theta_f32 = false;
        L.timeout_ns = 20000000000ull;
        L.stream = st;
        LaunchResult r;
        rc = run_plain(L, &r);
        if (rc == SP_OK) rc = map_device_error(r.err, "sigma", r.diag);
    }
    cudaError_t e = cudaSuccess;
    if (rc == SP_OK && host_m) e = cudaMemcpyAsync(mant_out, d_m, sizeof(double) * n, cudaMemcpyDeviceToHost, st);
    if (rc == SP_OK && e == cudaSuccess && host_e)
        e = cudaMemcpyAsync(exp2_out, d_e, sizeof(long long) * n, cudaMemcpyDeviceToHost, st);
    if (e != cudaSuccess) rc = cuda_fail(e, "copying sigma");
    if (d_src) cudaFreeAsync(d_src, st);
    if (host_m) cudaFreeAsync(d_m, st);
    if (host_e) cudaFreeAsync(d_e, st);
    e = cudaStreamSynchronize(st);
    if (rc == SP_OK && e != cudaSuccess) rc = cuda_fail(e, "sp_sigma");
    return rc;
}

}  // extern "C"
