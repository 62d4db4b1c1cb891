// Small-graph form: one thread block per source, every per-source array in
// shared memory.
//
// For graphs whose per-vertex state fits in one block's shared memory (16 B
// per vertex: level, a slot holding sigma and then theta, and the level
// stack), each block runs whole sources on its own (paper Section 2, Fig. 1,
// ComputeBC; level-synchronous BFS of Section 3.4) with __syncthreads as the
// level barrier, so a level costs shared-memory latency instead of a grid
// barrier and global round trips.  The CSR is read through the caches.
//
//   forward   entries of level d (the level stack, in shared memory) pull
//             sigma from neighbours at level d-1 and claim unvisited
//             neighbours for level d+1 (shared-memory atomicCAS), one lane per
//             row of at most 32 arcs, the whole warp for longer rows
//   backward  for d = L-1 ... 1 the entries of level d sum theta(w) =
//             (1 + delta(w)) / sigma(w) over neighbours at level d+1, then
//             delta(v) = sigma(v) * sum; theta(v) overwrites sigma(v) in the
//             same slot (sigma(v) is not read again); delta(v) is added to
//             the block's partial BC row
// Blocks take sources blockIdx.x, blockIdx.x + gridDim.x, ...; the partial
// rows are added in block order afterwards.  Every per-vertex sum runs in
// CSR order: results are bit-identical from run to run on a given GPU.
// Path counts are exact u64 sums; a carry stops the call with
// kErrSigmaOverflow and the host reruns it in another form.
#include <algorithm>
#include <climits>
#include <cstring>
#include <mutex>
#include <string>
#include <type_traits>

#include "common.cuh"
#include "internal.h"

namespace sp {

constexpr int kSmallThreads = 512;  // largest block; small graphs use 256 (below)
#ifndef SP_SMALL_BLOCK_MAXN
#define SP_SMALL_BLOCK_MAXN 3500
#endif

struct SmallArgs {
    const int32_t* rp;
    const int32_t* ci;
    int32_t n;
    const int32_t* sources;
    int32_t nsrc;
    double* bcpart;   // [gridDim.x][n] partial BC per block
    int32_t* qoff;    // [gridDim.x][n + 2] level offsets per block
    Ctl* ctl;
    const int* pre_err;  // asynchronous calls: nonzero = the sources failed their check, do nothing
    int directed;        // rp/ci: combined out- and in-arc rows (arc_in / arc_out); odeg: out-degrees
    const int32_t* odeg;
};

// Shared-memory bytes of one block for n vertices.
inline size_t small_smem_bytes(int64_t n) { return (size_t)n * 16 + 64; }

template <typename ThT>
__global__ void __launch_bounds__(kSmallThreads, 2) small_kernel(SmallArgs a) {
    if (a.pre_err != nullptr) {
        const int pe = ld_volatile(a.pre_err);
        if (pe != 0) {
            if (blockIdx.x == 0 && threadIdx.x == 0) a.ctl->err = pe;
            return;
        }
    }
    extern __shared__ __align__(16) unsigned char smem[];
    const int n = a.n;
    unsigned long long* slot = reinterpret_cast<unsigned long long*>(smem);  // sigma, then theta bits
    int32_t* lvl = reinterpret_cast<int32_t*>(smem + (size_t)n * 8);
    int32_t* q = lvl + n;
    __shared__ int s_qtail;
    __shared__ int s_err;
    __shared__ unsigned long long s_st[4];

    const int tid = threadIdx.x;
    const int lane = tid & 31;
    const int warp = tid >> 5;
    const int nwarps = blockDim.x >> 5;
    double* bcp = a.bcpart + (size_t)blockIdx.x * (size_t)n;
    int32_t* qoff = a.qoff + (size_t)blockIdx.x * (size_t)(n + 2);
    unsigned long long st_arcs = 0, st_reached = 0, st_scanned = 0, st_dag = 0;
    int levels_max = 0;
    if (tid == 0) s_err = 0;
    for (int i = tid; i < n; i += blockDim.x) bcp[i] = 0.0;

    auto theta_of = [&](int w) -> double {
        if constexpr (sizeof(ThT) == 4) {
            return (double)__uint_as_float((unsigned)slot[w]);
        } else {
            return __longlong_as_double((long long)slot[w]);
        }
    };

    for (int si = blockIdx.x; si < a.nsrc; si += gridDim.x) {
        const int src = __ldg(&a.sources[si]);
        __syncthreads();
        for (int i = tid; i < n; i += blockDim.x) lvl[i] = -1;
        __syncthreads();
        if (tid == 0) {
            lvl[src] = 0;
            slot[src] = 1ull;
            q[0] = src;
            s_qtail = 1;
            qoff[0] = 0;
            qoff[1] = 1;
        }
        __syncthreads();

        // ---- forward ----
        int qb = 0, qe = 1, d = 0;
        bool ovf = false;
        while (true) {
            // entries [qb, qe) of level d, 32 per warp at a time, lane per entry
            for (int e0 = qb + warp * 32; e0 < qe; e0 += nwarps * 32) {
                const int e = e0 + lane;
                const bool valid = e < qe;
                const int v = valid ? q[e] : 0;
                int beg = 0, deg = 0;
                if (valid) {
                    beg = __ldg(&a.rp[v]);
                    deg = __ldg(&a.rp[v + 1]) - beg;
                    st_arcs += (unsigned long long)(a.odeg != nullptr ? __ldg(&a.odeg[v]) : deg);
                    st_reached += 1;
                    st_scanned += (unsigned long long)deg;
                }
                unsigned long long acc = 0;
                // arc `raw` of v: claim its other end over an arc out of v, or
                // take its path count over an arc into v from level d-1
                auto visit = [&](int raw) -> unsigned long long {
                    const int u = arc_vertex(raw);
                    const int lu = lvl[u];
                    if (lu < 0) {
                        if (arc_out(raw) && atomicCAS(&lvl[u], -1, d + 1) == -1) q[atomicAdd(&s_qtail, 1)] = u;
                    } else if (lu == d - 1 && arc_in(raw, a.directed)) {
                        st_dag += 1;
                        return slot[u];
                    }
                    return 0ull;
                };
                if (deg <= 32) {
                    // column ids eight at a time (independent cached loads), then
                    // the shared-memory visits in CSR order
                    for (int k0 = 0; k0 < deg; k0 += 8) {
                        int u[8];
#pragma unroll
                        for (int i = 0; i < 8; ++i) u[i] = k0 + i < deg ? __ldg(&a.ci[beg + k0 + i]) : 0;
#pragma unroll
                        for (int i = 0; i < 8; ++i) {
                            if (k0 + i >= deg) continue;
                            const unsigned long long c = visit(u[i]);
                            const unsigned long long s = acc + c;
                            ovf |= s < acc;
                            acc = s;
                        }
                    }
                }
                unsigned big = __ballot_sync(kFull, deg > 32);
                while (big) {
                    const int j = __ffs(big) - 1;
                    big &= big - 1;
                    const int bj = __shfl_sync(kFull, beg, j), dj = __shfl_sync(kFull, deg, j);
                    unsigned long long p = 0;
                    for (int k = lane; k < dj; k += 32) {
                        const unsigned long long c = visit(__ldg(&a.ci[bj + k]));
                        const unsigned long long s = p + c;
                        ovf |= s < p;
                        p = s;
                    }
                    for (int o = 16; o > 0; o >>= 1) {
                        const unsigned long long y = shfl_u64(kFull, p, lane ^ o);
                        const unsigned long long s = p + y;
                        ovf |= s < p;
                        p = s;
                    }
                    if (lane == j) acc = p;
                }
                if (valid && d > 0) slot[v] = acc;
            }
            if (ovf) s_err = kErrSigmaOverflow;
            __syncthreads();
            const int nq = s_qtail;
            __syncthreads();  // every thread has read the fill before level d+1 pushes
            if (s_err != 0) break;
            if (nq == qe) break;
            qb = qe;
            qe = nq;
            ++d;
            if (tid == 0) qoff[d + 1] = qe;
        }
        if (s_err != 0) break;
        const int L = d + 1;
        levels_max = max(levels_max, L);
        __syncthreads();  // qoff[] written by thread 0

        // ---- backward ----
        for (int dd = L - 1; dd >= 1; --dd) {
            const int b = qoff[dd], e1 = qoff[dd + 1];
            const bool leaf_level = dd == L - 1;
            for (int e0 = b + warp * 32; e0 < e1; e0 += nwarps * 32) {
                const int e = e0 + lane;
                const bool valid = e < e1;
                const int v = valid ? q[e] : 0;
                int beg = 0, deg = 0;
                if (valid && !leaf_level) {
                    beg = __ldg(&a.rp[v]);
                    deg = __ldg(&a.rp[v + 1]) - beg;
                    st_scanned += (unsigned long long)deg;
                }
                double acc = 0.0;
                if (deg <= 32) {
                    for (int k0 = 0; k0 < deg; k0 += 8) {
                        int w[8];
#pragma unroll
                        for (int i = 0; i < 8; ++i) w[i] = k0 + i < deg ? __ldg(&a.ci[beg + k0 + i]) : -1;
#pragma unroll
                        for (int i = 0; i < 8; ++i)  // children: out-arcs (an in-arc is negative here)
                            if (w[i] >= 0 && lvl[w[i]] == dd + 1) acc += theta_of(w[i]);
                    }
                }
                unsigned big = __ballot_sync(kFull, deg > 32);
                while (big) {
                    const int j = __ffs(big) - 1;
                    big &= big - 1;
                    const int bj = __shfl_sync(kFull, beg, j), dj = __shfl_sync(kFull, deg, j);
                    double p = 0.0;
                    for (int k = lane; k < dj; k += 32) {
                        const int w = __ldg(&a.ci[bj + k]);
                        if (arc_out(w) && lvl[w] == dd + 1) p += theta_of(w);
                    }
                    p = warp_sum_f64(p);
                    if (lane == j) acc = p;
                }
                if (valid) {
                    const double sv = (double)slot[v];
                    const double delta = sv * acc;
                    const double t = (1.0 + delta) / sv;
                    if constexpr (sizeof(ThT) == 4) {
                        const float tf = (float)t;
                        if (!normal_finite_f(tf)) s_err = kErrThetaRange32;
                        slot[v] = (unsigned long long)__float_as_uint(tf);
                    } else {
                        if (!normal_finite(t)) s_err = SP_ERR_RANGE;
                        slot[v] = (unsigned long long)__double_as_longlong(t);
                    }
                    bcp[v] += delta;
                }
            }
            __syncthreads();
        }
        if (s_err != 0) break;
    }

    // statistics and errors
    __syncthreads();
    if (tid == 0) { s_st[0] = 0; s_st[1] = 0; s_st[2] = 0; s_st[3] = 0; }
    __syncthreads();
    atomicAdd(&s_st[0], st_arcs);
    atomicAdd(&s_st[1], st_reached);
    atomicAdd(&s_st[2], st_scanned);
    atomicAdd(&s_st[3], st_dag);
    __syncthreads();
    if (tid == 0) {
        atomicAdd(&a.ctl->traversed_arcs, s_st[0]);
        atomicAdd(&a.ctl->reached, s_st[1]);
        atomicAdd(&a.ctl->entries, s_st[1]);
        atomicAdd(&a.ctl->scanned_arcs, s_st[2]);
        atomicAdd(&a.ctl->dag_arcs, s_st[3]);
        atomicMax(&a.ctl->max_levels, levels_max);
        if (s_err != 0) set_error(a.ctl, s_err);
    }
}

// Sum of the blocks' partial BC rows, in block order.
static __global__ void small_sum_kernel(const double* __restrict__ part, int nparts, int64_t n,
                                        double* __restrict__ out) {
    for (int64_t v = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; v < n; v += (int64_t)gridDim.x * blockDim.x) {
        double s = 0.0;
        for (int b = 0; b < nparts; ++b) s += part[(int64_t)b * n + v];
        out[v] = s;
    }
}

int64_t small_form_max_n(int device) {
    static int64_t cache[64] = {0};
    if (device < 0 || device >= 64) return 0;
    if (cache[device] == 0) {
        int optin = 0;
        if (cudaDeviceGetAttribute(&optin, cudaDevAttrMaxSharedMemoryPerBlockOptin, device) != cudaSuccess) {
            cudaGetLastError();
            return 0;
        }
        // the kernel's static shared memory is a few dozen bytes
        cache[device] = std::max<int64_t>(1, ((int64_t)optin - 256 - 64) / 16);
    }
    return cache[device];
}

sp_status run_small(const SmallLaunch& L, LaunchResult* result) {
    const Graph* g = L.g;
    const int64_t n = g->n;
    cudaStream_t st = L.stream;
    if (n > small_form_max_n(g->device)) return fail(SP_ERR_TOO_LARGE, "graph too large for the small form");
    const void* fn = L.theta_f32 ? (const void*)&small_kernel<float> : (const void*)&small_kernel<double>;
    const size_t smem = small_smem_bytes(n);
    {
        // Raise the kernels' dynamic shared-memory limit once per device to
        // the largest size any graph of this form needs (never per call:
        // calls on other host threads may be launching with larger sizes).
        static std::mutex mu;
        static bool done[64] = {false};
        std::lock_guard<std::mutex> lk(mu);
        const int dev = g->device;
        if (dev < 0 || dev >= 64) return fail(SP_ERR_INVALID_ARG, "device id");
        if (!done[dev]) {
            const int lim = (int)small_smem_bytes(small_form_max_n(dev));
            SP_CUDA(cudaFuncSetAttribute((const void*)&small_kernel<float>, cudaFuncAttributeMaxDynamicSharedMemorySize, lim));
            SP_CUDA(cudaFuncSetAttribute((const void*)&small_kernel<double>, cudaFuncAttributeMaxDynamicSharedMemorySize, lim));
            done[dev] = true;
        }
    }
    int per_sm = 0;
    // Blocks of 256 threads when four fit an SM's shared memory (more sources
    // side by side; a level of a graph this small rarely needs more warps),
    // else 512.
    const int threads = n <= SP_SMALL_BLOCK_MAXN ? 256 : kSmallThreads;
    SP_CUDA(cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, fn, threads, smem));
    if (per_sm < 1) return fail(SP_ERR_TOO_LARGE, "small form cannot be resident");
    int grid = per_sm * device_sm_count(g->device);
    if (L.max_ctas > 0 && L.max_ctas < grid) grid = L.max_ctas;
    grid = std::max(1, std::min(grid, L.nsrc));

    size_t bytes = 0;
    auto take = [&](size_t b) { size_t o = bytes; bytes += (b + 255) & ~(size_t)255; return o; };
    const size_t o_ctl = take(sizeof(Ctl));
    const size_t o_part = take(sizeof(double) * (size_t)n * grid);
    const size_t o_qoff = take(sizeof(int32_t) * (size_t)(n + 2) * grid);
    char* ws = nullptr;
    if (workspace_alloc((void**)&ws, bytes, st) != cudaSuccess) {
        cudaGetLastError();
        return fail(SP_ERR_OOM, "workspace allocation (small form)");
    }
    struct FreeWs {
        char* p;
        cudaStream_t s;
        ~FreeWs() { cudaFreeAsync(p, s); }
    } free_ws{ws, st};
    SP_CUDA(cudaMemsetAsync(ws, 0, sizeof(Ctl), st));

    SmallArgs a{};
    a.rp = g->krp();
    a.ci = g->kci();
    a.directed = g->directed;
    a.odeg = g->d_odeg;
    a.n = (int32_t)n;
    a.sources = L.d_sources;
    a.nsrc = L.nsrc;
    a.bcpart = reinterpret_cast<double*>(ws + o_part);
    a.qoff = reinterpret_cast<int32_t*>(ws + o_qoff);
    a.ctl = reinterpret_cast<Ctl*>(ws + o_ctl);
    a.pre_err = L.async.pre_err;

    if (L.async.flags != nullptr) {  // enqueue only: the finish step moves the error word on
        void* args[] = {&a};
        cudaError_t ce = cudaLaunchKernel(fn, dim3(grid), dim3(threads), args, smem, st);
        if (ce == cudaSuccess) {
            const int rgrid = (int)std::min<int64_t>((n + 255) / 256, (int64_t)device_sm_count(g->device) * 8);
            small_sum_kernel<<<std::max(rgrid, 1), 256, 0, st>>>(a.bcpart, grid, n, L.d_bc);
            ce = cudaGetLastError();
        }
        if (ce != cudaSuccess) return cuda_fail(ce, "small form");
        result->launches = 3;
        result->grid = grid;
        result->groups = grid;
        return enqueue_finish(a.ctl, L.async, st);  // the workspace is freed after it (FreeWs)
    }

    cudaEvent_t ev0, ev1;
    cudaEventCreate(&ev0);
    cudaEventCreate(&ev1);
    cudaEventRecord(ev0, st);
    void* args[] = {&a};
    cudaError_t ce = cudaLaunchKernel(fn, dim3(grid), dim3(threads), args, smem, st);
    if (ce == cudaSuccess) {
        const int rgrid = (int)std::min<int64_t>((n + 255) / 256, (int64_t)device_sm_count(g->device) * 8);
        small_sum_kernel<<<std::max(rgrid, 1), 256, 0, st>>>(a.bcpart, grid, n, L.d_bc);
        ce = cudaGetLastError();
    }
    cudaEventRecord(ev1, st);
    static thread_local Ctl h;
    std::memset(&h, 0, sizeof(h));
    if (ce == cudaSuccess) ce = cudaMemcpyAsync(&h, ws + o_ctl, sizeof(Ctl), cudaMemcpyDeviceToHost, st);
    if (ce == cudaSuccess) ce = cudaStreamSynchronize(st);
    float ms = 0.0f;
    if (ce == cudaSuccess && cudaEventElapsedTime(&ms, ev0, ev1) == cudaSuccess) result->kernel_ms = ms;
    cudaEventDestroy(ev0);
    cudaEventDestroy(ev1);
    if (ce != cudaSuccess) return cuda_fail(ce, "small form");
    result->err = h.err;
    result->levels = h.max_levels;
    result->traversed_arcs = h.traversed_arcs;
    result->reached = h.reached;
    result->entries = h.entries;
    result->scanned_arcs = h.scanned_arcs;
    result->dag_arcs = h.dag_arcs;
    result->grid = grid;
    result->groups = grid;
    result->launches = 2;
    return SP_OK;
}

}  // namespace sp
