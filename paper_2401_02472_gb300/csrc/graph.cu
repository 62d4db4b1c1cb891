// CSR validation and degree statistics on the GPU (graph construction step).
//
// The paper keeps the graph as a CSR offset array plus edge list, copied to
// the device once and kept there while properties change (Section 3.1 and the
// host-device transfer optimisation of Section 4.1).  Here the copy is checked
// on the device before any traversal uses it.
#include <climits>
#include <mutex>

#include "common.cuh"
#include "internal.h"

namespace sp {

struct ValidateOut {
    int bad_rowptr;        // first v with row_ptr[v] > row_ptr[v+1], or INT_MAX
    int bad_col;           // first arc index with col out of range, or INT_MAX
    int max_degree;
    int unsorted;          // 1 if some row is not strictly increasing
    int self_loops;
    int duplicates;
    int asymmetric;        // 1 if some arc has no reverse (symmetric check only)
    unsigned long long isolated;
    unsigned long long top;  // (max degree << 32) | ~vertex: the smallest-id vertex of maximum degree
};

__global__ void rowptr_kernel(const int32_t* __restrict__ rp, int32_t n, int64_t nnz, ValidateOut* out) {
    int v = blockIdx.x * blockDim.x + threadIdx.x;
    int maxdeg = 0;
    unsigned long long iso = 0, top = 0;
    for (; v < n; v += gridDim.x * blockDim.x) {
        int a = rp[v], b = rp[v + 1];
        if (b < a || a < 0 || (int64_t)b > nnz) atomicMin(&out->bad_rowptr, v);
        int dg = b - a;
        maxdeg = max(maxdeg, dg);
        iso += dg == 0;
        unsigned long long key = ((unsigned long long)(unsigned)max(dg, 0) << 32) | (unsigned)(~(unsigned)v);
        top = key > top ? key : top;
    }
    maxdeg = warp_max_i32(maxdeg);
    iso = warp_sum_u64(iso);
    for (int o = 16; o > 0; o >>= 1) {
        unsigned long long y = shfl_u64(kFull, top, lane_id() ^ o);
        top = y > top ? y : top;
    }
    if ((threadIdx.x & 31) == 0) {
        atomicMax(&out->max_degree, maxdeg);
        atomicAdd(&out->isolated, iso);
        atomicMax(&out->top, top);
    }
}

// Ids in range, strict order, self-loops, repeats.  A warp takes 32
// consecutive rows: a lane walks its own row when it has at most 32 arcs
// (most rows of sparse graphs), the whole warp walks each longer row.
__global__ void rows_kernel(const int32_t* __restrict__ rp, const int32_t* __restrict__ ci, int32_t n,
                            ValidateOut* out) {
    const int lane = threadIdx.x & 31;
    const int warp = (blockIdx.x * blockDim.x + threadIdx.x) >> 5;
    const int nwarp = (gridDim.x * blockDim.x) >> 5;
    bool unsorted = false, loop = false, dup = false;
    for (int64_t v0 = (int64_t)warp * 32; v0 < n; v0 += (int64_t)nwarp * 32) {
        const int v = (int)(v0 + lane);
        int a = 0, b = 0;
        if (v < n) { a = rp[v]; b = rp[v + 1]; }
        const bool mine = b - a <= 32;
        if (v < n && mine) {
            int prev = INT_MIN;
            for (int e = a; e < b; ++e) {
                const int c = ci[e];
                if (c < 0 || c >= n) { atomicMin(&out->bad_col, e); prev = INT_MIN; continue; }
                loop |= c == v;
                if (prev != INT_MIN) { unsorted |= c <= prev; dup |= c == prev; }
                prev = c;
            }
        }
        unsigned big = __ballot_sync(kFull, v < n && !mine);
        while (big) {
            const int j = __ffs(big) - 1;
            big &= big - 1;
            const int vj = (int)(v0 + j);
            const int aj = __shfl_sync(kFull, a, j), bj = __shfl_sync(kFull, b, j);
            // eight coalesced loads per lane in flight: a hub row of 10^5
            // arcs is not a chain of 3,000 dependent loads
            for (int e0 = aj; e0 < bj; e0 += 8 * 32) {
                int c[8], c2[8];
#pragma unroll
                for (int k = 0; k < 8; ++k) {
                    const int e = e0 + k * 32 + lane;
                    c[k] = e < bj ? ci[e] : 0;
                    c2[k] = e + 1 < bj ? ci[e + 1] : 0;
                }
#pragma unroll
                for (int k = 0; k < 8; ++k) {
                    const int e = e0 + k * 32 + lane;
                    if (e >= bj) continue;
                    if (c[k] < 0 || c[k] >= n) { atomicMin(&out->bad_col, e); continue; }
                    loop |= c[k] == vj;
                    if (e + 1 < bj) {
                        unsorted |= c2[k] <= c[k];
                        dup |= c2[k] == c[k];
                    }
                }
            }
        }
    }
    if (__any_sync(kFull, unsorted) && lane == 0) out->unsorted = 1;
    if (__any_sync(kFull, loop) && lane == 0) out->self_loops = 1;
    if (__any_sync(kFull, dup) && lane == 0) out->duplicates = 1;
}

// One warp per row: every arc (v, c) must have its reverse (c, v); rows sorted.
__global__ void symmetric_kernel(const int32_t* __restrict__ rp, const int32_t* __restrict__ ci, int32_t n,
                                 ValidateOut* out) {
    const int lane = threadIdx.x & 31;
    const int warp = (blockIdx.x * blockDim.x + threadIdx.x) >> 5;
    const int nwarp = (gridDim.x * blockDim.x) >> 5;
    for (int v = warp; v < n; v += nwarp) {
        int a = rp[v], b = rp[v + 1];
        bool miss = false;
        for (int e = a + lane; e < b; e += 32) {
            int c = ci[e];
            int lo = rp[c], hi = rp[c + 1];
            while (lo < hi) {
                int mid = (lo + hi) >> 1;
                if (ci[mid] < v) lo = mid + 1; else hi = mid;
            }
            miss |= !(lo < rp[c + 1] && ci[lo] == v);
        }
        if (__any_sync(kFull, miss) && lane == 0) out->asymmetric = 1;
    }
}

// Launch workspaces come from a memory pool of the library's own that keeps
// freed memory (release threshold: unlimited), so that a call does not map
// gigabytes of fresh memory because an earlier call's workspace went back to
// the device between them.  A failed allocation trims the pool and retries.
cudaError_t workspace_alloc(void** p, size_t bytes, cudaStream_t st) {
    static std::mutex mu;
    static cudaMemPool_t pools[64] = {};
    static bool failed[64] = {};
    int dev = 0;
    cudaError_t e = cudaGetDevice(&dev);
    if (e != cudaSuccess || dev < 0 || dev >= 64) return cudaMallocAsync(p, bytes, st);
    cudaMemPool_t pool = nullptr;
    {
        std::lock_guard<std::mutex> lk(mu);
        if (!pools[dev] && !failed[dev]) {
            cudaMemPoolProps props{};
            props.allocType = cudaMemAllocationTypePinned;
            props.handleTypes = cudaMemHandleTypeNone;
            props.location.type = cudaMemLocationTypeDevice;
            props.location.id = dev;
            if (cudaMemPoolCreate(&pools[dev], &props) == cudaSuccess) {
                uint64_t keep = ~0ull;
                cudaMemPoolSetAttribute(pools[dev], cudaMemPoolAttrReleaseThreshold, &keep);
            } else {
                cudaGetLastError();
                pools[dev] = nullptr;
                failed[dev] = true;
            }
        }
        pool = pools[dev];
    }
    if (!pool) return cudaMallocAsync(p, bytes, st);
    e = cudaMallocFromPoolAsync(p, bytes, pool, st);
    if (e == cudaErrorMemoryAllocation) {
        cudaGetLastError();
        cudaStreamSynchronize(st);
        cudaMemPoolTrimTo(pool, 0);
        e = cudaMallocFromPoolAsync(p, bytes, pool, st);
    }
    return e;
}

int device_sm_count(int device) {
    static int cache[64] = {0};
    if (device < 0 || device >= 64) return 1;
    if (cache[device] == 0) {
        int c = 0;
        cudaDeviceGetAttribute(&c, cudaDevAttrMultiProcessorCount, device);
        cache[device] = c > 0 ? c : 1;
    }
    return cache[device];
}

sp_status validate_graph(Graph* g, uint32_t flags, cudaStream_t st, std::string* detail) {
    ValidateOut h{};
    h.bad_rowptr = INT_MAX;
    h.bad_col = INT_MAX;
    ValidateOut* d = nullptr;
    SP_CUDA(cudaMallocAsync((void**)&d, sizeof(ValidateOut), st));
    cudaError_t ce = cudaMemcpyAsync(d, &h, sizeof(h), cudaMemcpyHostToDevice, st);
    const int sms = device_sm_count(g->device);
    int32_t first = 0, last = 0;
    if (ce == cudaSuccess) ce = cudaMemcpyAsync(&first, g->d_rp, sizeof(int32_t), cudaMemcpyDeviceToHost, st);
    if (ce == cudaSuccess)
        ce = cudaMemcpyAsync(&last, g->d_rp + g->n, sizeof(int32_t), cudaMemcpyDeviceToHost, st);
    if (ce == cudaSuccess && g->n > 0) {
        rowptr_kernel<<<sms * 4, 256, 0, st>>>(g->d_rp, g->n, g->nnz, d);
        ce = cudaGetLastError();
    }
    if (ce == cudaSuccess) ce = cudaMemcpyAsync(&h, d, sizeof(h), cudaMemcpyDeviceToHost, st);
    if (ce == cudaSuccess) ce = cudaStreamSynchronize(st);
    if (ce != cudaSuccess) { cudaFreeAsync(d, st); return cuda_fail(ce, "row_ptr validation"); }
    if (first != 0 || (int64_t)last != g->nnz || h.bad_rowptr != INT_MAX) {
        cudaFreeAsync(d, st);
        if (first != 0) *detail = "row_ptr[0] != 0";
        else if ((int64_t)last != g->nnz) *detail = "row_ptr[n] != nnz";
        else *detail = "row_ptr decreases or leaves [0, nnz] at row " + std::to_string(h.bad_rowptr);
        return SP_ERR_BAD_GRAPH;
    }
    if (g->n > 0 && g->nnz > 0) {
        rows_kernel<<<sms * 8, 256, 0, st>>>(g->d_rp, g->d_ci, g->n, d);
        ce = cudaGetLastError();
        if (ce == cudaSuccess) ce = cudaMemcpyAsync(&h, d, sizeof(h), cudaMemcpyDeviceToHost, st);
        if (ce == cudaSuccess) ce = cudaStreamSynchronize(st);
        if (ce != cudaSuccess) { cudaFreeAsync(d, st); return cuda_fail(ce, "col_idx validation"); }
        if (h.bad_col != INT_MAX) {
            cudaFreeAsync(d, st);
            *detail = "col_idx out of [0, n) at arc " + std::to_string(h.bad_col);
            return SP_ERR_BAD_GRAPH;
        }
    }
    g->info.n = g->n;
    g->info.nnz = g->nnz;
    g->info.max_degree = h.max_degree;
    g->top_vertex = g->n > 0 ? (int32_t)(~(unsigned)(h.top & 0xFFFFFFFFull)) : 0;
    g->info.isolated = (int64_t)h.isolated;
    g->info.sorted_rows = h.unsorted ? 0 : 1;
    g->info.has_self_loops = h.self_loops;
    g->info.has_duplicates = h.duplicates;
    g->info.symmetric = -1;
    if (flags & SP_GRAPH_CHECK_SYMMETRIC) {
        if (h.unsorted) {
            cudaFreeAsync(d, st);
            *detail = "the symmetry check needs rows sorted by neighbour id";
            return SP_ERR_BAD_GRAPH;
        }
        if (g->n > 0 && g->nnz > 0) {
            symmetric_kernel<<<sms * 8, 256, 0, st>>>(g->d_rp, g->d_ci, g->n, d);
            ce = cudaGetLastError();
            if (ce == cudaSuccess) ce = cudaMemcpyAsync(&h, d, sizeof(h), cudaMemcpyDeviceToHost, st);
            if (ce == cudaSuccess) ce = cudaStreamSynchronize(st);
            if (ce != cudaSuccess) { cudaFreeAsync(d, st); return cuda_fail(ce, "symmetry check"); }
        }
        g->info.symmetric = h.asymmetric ? 0 : 1;
        if (h.asymmetric) {
            cudaFreeAsync(d, st);
            *detail = "some arc (u, v) has no reverse arc (v, u)";
            return SP_ERR_BAD_GRAPH;
        }
    }
    cudaFreeAsync(d, st);
    return SP_OK;
}

}  // namespace sp
