// CSR construction on the GPU: sorting rows, and building a symmetric,
// deduplicated CSR from an edge list.
//
// The paper's graphs arrive as edge lists and are turned into the CSR offset
// array + edge list that every backend reads (Section 3.1, graph
// representation); here that step runs on the device.
//
//   row sort        rows of 2..32 arcs: one warp per row, a bitonic network
//                   across the lanes; 33..4096 arcs: one block per row, a
//                   bitonic network in shared memory; longer rows: 4096-arc
//                   pieces sorted the same way, then merged pairwise (each
//                   element finds its place by binary search in the partner
//                   run, ties to the left run), doubling the run length.
//   edge list       both arcs of every edge that is not a self-loop are
//                   counted per row, offsets come from an exclusive scan, the
//                   arcs are scattered into their rows, the rows are sorted,
//                   and repeats within a row are dropped (count, scan, compact).
// Every step is deterministic: the output depends only on the input multiset.
#include <algorithm>
#include <climits>
#include <cstring>
#include <string>
#include <vector>

#include "common.cuh"
#include "internal.h"

namespace sp {

namespace {

constexpr int kSortTile = 4096;  // longest row one block sorts in shared memory

__device__ __forceinline__ int next_pow2(int x) {
    int p = 1;
    while (p < x) p <<= 1;
    return p;
}

// Rows of at least two arcs, by length class.
__global__ void classify_rows_kernel(const int32_t* __restrict__ rp, int32_t n, int32_t* __restrict__ cnt,
                                     int32_t* __restrict__ small, int32_t* __restrict__ mid,
                                     int32_t* __restrict__ big) {
    for (int v = blockIdx.x * blockDim.x + threadIdx.x; v < n; v += gridDim.x * blockDim.x) {
        const int d = rp[v + 1] - rp[v];
        if (d < 2) continue;
        if (d <= 32) small[atomicAdd(&cnt[0], 1)] = v;
        else if (d <= kSortTile) mid[atomicAdd(&cnt[1], 1)] = v;
        else big[atomicAdd(&cnt[2], 1)] = v;
    }
}

// One warp per row of at most 32 arcs: bitonic sort across the lanes.
__global__ void sort_rows_warp_kernel(const int32_t* __restrict__ rp, int32_t* __restrict__ ci,
                                      const int32_t* __restrict__ rows, int32_t count) {
    const int lane = threadIdx.x & 31;
    const int warp = (blockIdx.x * blockDim.x + threadIdx.x) >> 5;
    const int nwarp = (gridDim.x * blockDim.x) >> 5;
    for (int r = warp; r < count; r += nwarp) {
        const int v = rows[r];
        const int b = rp[v], d = rp[v + 1] - b;
        int x = lane < d ? ci[b + lane] : INT_MAX;
#pragma unroll
        for (int k = 2; k <= 32; k <<= 1) {
#pragma unroll
            for (int j = k >> 1; j > 0; j >>= 1) {
                const int y = __shfl_xor_sync(kFull, x, j);
                const bool up = (lane & k) == 0;
                const bool low = (lane & j) == 0;
                x = (low == up) ? min(x, y) : max(x, y);
            }
        }
        if (lane < d) ci[b + lane] = x;
    }
}

// One block per segment [seg.x, seg.y) of at most kSortTile arcs: bitonic
// sort in shared memory, padded to a power of two with INT_MAX.
__global__ void sort_segments_block_kernel(int32_t* __restrict__ ci, const int2* __restrict__ segs, int32_t count) {
    __shared__ int s[kSortTile];
    for (int r = blockIdx.x; r < count; r += gridDim.x) {
        const int b = segs[r].x, d = segs[r].y - segs[r].x;
        const int P = next_pow2(d);
        __syncthreads();
        for (int i = threadIdx.x; i < P; i += blockDim.x) s[i] = i < d ? ci[b + i] : INT_MAX;
        __syncthreads();
        for (int k = 2; k <= P; k <<= 1) {
            for (int j = k >> 1; j > 0; j >>= 1) {
                for (int i = threadIdx.x; i < P; i += blockDim.x) {
                    const int p = i ^ j;
                    if (p > i) {
                        const int a = s[i], c = s[p];
                        const bool up = (i & k) == 0;
                        if ((a > c) == up) { s[i] = c; s[p] = a; }
                    }
                }
                __syncthreads();
            }
        }
        for (int i = threadIdx.x; i < d; i += blockDim.x) ci[b + i] = s[i];
    }
}

// Lower / upper bound of x in a[0, len).
__device__ __forceinline__ int lower_bound_i(const int32_t* a, int len, int x) {
    int lo = 0, hi = len;
    while (lo < hi) {
        const int mid = (lo + hi) >> 1;
        if (a[mid] < x) lo = mid + 1; else hi = mid;
    }
    return lo;
}
__device__ __forceinline__ int upper_bound_i(const int32_t* a, int len, int x) {
    int lo = 0, hi = len;
    while (lo < hi) {
        const int mid = (lo + hi) >> 1;
        if (a[mid] <= x) lo = mid + 1; else hi = mid;
    }
    return lo;
}

// One merge pass over long rows: runs of `run` sorted arcs are merged in
// pairs.  Row r occupies src[row.x, row.y) and dst[off, off + len) with off
// given per row (the two buffers need not share offsets).
__global__ void merge_pass_kernel(const int32_t* __restrict__ src, const int64_t* __restrict__ src_off,
                                  int32_t* __restrict__ dst, const int64_t* __restrict__ dst_off,
                                  const int32_t* __restrict__ lens, int32_t nrows, int run) {
    for (int r = blockIdx.x; r < nrows; r += gridDim.x) {
        const int32_t* a = src + src_off[r];
        int32_t* o = dst + dst_off[r];
        const int len = lens[r];
        for (int i = threadIdx.x; i < len; i += blockDim.x) {
            const int64_t span = 2 * (int64_t)run;
            const int lb = (int)((i / span) * span);
            const int mid = (int)min((int64_t)lb + run, (int64_t)len), hb = (int)min((int64_t)lb + span, (int64_t)len);
            const int x = a[i];
            int pos;
            if (i < mid) pos = lb + (i - lb) + lower_bound_i(a + mid, hb - mid, x);
            else pos = lb + (i - mid) + upper_bound_i(a + lb, mid - lb, x);
            o[pos] = x;
        }
    }
}

__global__ void gather_rows_kernel(const int32_t* __restrict__ rp, const int32_t* __restrict__ rows, int32_t count,
                                   int2* __restrict__ out) {
    for (int r = blockIdx.x * blockDim.x + threadIdx.x; r < count; r += gridDim.x * blockDim.x)
        out[r] = make_int2(rp[rows[r]], rp[rows[r] + 1]);
}

// Block-wise exclusive scan of `in` (count values): out[i] = sum of the
// block's values before i; sums[b] = the block's total.
constexpr int kScanBlock = 1024;
__global__ void scan_blocks_kernel(const int32_t* __restrict__ in, int64_t count, int32_t* __restrict__ out,
                                   int32_t* __restrict__ sums) {
    __shared__ int warp_tot[kScanBlock / 32];
    const int64_t i = (int64_t)blockIdx.x * kScanBlock + threadIdx.x;
    const int x = i < count ? in[i] : 0;
    const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
    const int incl = warp_incl_scan(x);
    if (lane == 31) warp_tot[w] = incl;
    __syncthreads();
    if (w == 0) {
        const int t = warp_incl_scan(warp_tot[lane]);
        warp_tot[lane] = t;
    }
    __syncthreads();
    const int base = w > 0 ? warp_tot[w - 1] : 0;
    if (i < count) out[i] = base + incl - x;
    if (threadIdx.x == kScanBlock - 1) sums[blockIdx.x] = base + incl;
}

__global__ void scan_add_kernel(int32_t* __restrict__ out, int64_t count, const int32_t* __restrict__ offs) {
    const int64_t i = (int64_t)blockIdx.x * kScanBlock + threadIdx.x;
    if (i < count) out[i] += offs[blockIdx.x];
}

// Edge list: endpoint check and per-row arc counts (both directions, no loops).
// Edge list: endpoint check and per-row arc counts (both directions, or only
// src -> dst for a directed graph; no loops).
__global__ void edge_count_kernel(const int32_t* __restrict__ src, const int32_t* __restrict__ dst, int64_t m,
                                  int32_t n, bool directed, int32_t* __restrict__ deg,
                                  unsigned long long* __restrict__ bad) {
    for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < m; i += (int64_t)gridDim.x * blockDim.x) {
        const int u = src[i], v = dst[i];
        if (u < 0 || u >= n || v < 0 || v >= n) { atomicMin(bad, (unsigned long long)i); continue; }
        if (u == v) continue;
        atomicAdd(&deg[u], 1);
        if (!directed) atomicAdd(&deg[v], 1);
    }
}

__global__ void edge_scatter_kernel(const int32_t* __restrict__ src, const int32_t* __restrict__ dst, int64_t m,
                                    bool directed, const int32_t* __restrict__ rp, int32_t* __restrict__ fill,
                                    int32_t* __restrict__ ci) {
    for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < m; i += (int64_t)gridDim.x * blockDim.x) {
        const int u = src[i], v = dst[i];
        if (u == v) continue;
        ci[rp[u] + atomicAdd(&fill[u], 1)] = v;
        if (!directed) ci[rp[v] + atomicAdd(&fill[v], 1)] = u;
    }
}

// Directed graphs: in-degree of every vertex (arc count per target).
__global__ void in_count_kernel(const int32_t* __restrict__ ci, int64_t nnz, int32_t* __restrict__ indeg) {
    for (int64_t e = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; e < nnz; e += (int64_t)gridDim.x * blockDim.x)
        atomicAdd(&indeg[ci[e]], 1);
}

// Directed graphs: the in-arc rows (warp per source row), in arrival order;
// sorted afterwards.
__global__ void in_scatter_kernel(const int32_t* __restrict__ rp, const int32_t* __restrict__ ci, int32_t n,
                                  const int32_t* __restrict__ irp, int32_t* __restrict__ fill,
                                  int32_t* __restrict__ ici) {
    const int lane = threadIdx.x & 31;
    const int warp = (blockIdx.x * blockDim.x + threadIdx.x) >> 5;
    const int nwarp = (gridDim.x * blockDim.x) >> 5;
    for (int u = warp; u < n; u += nwarp)
        for (int e = rp[u] + lane; e < rp[u + 1]; e += 32) {
            const int v = ci[e];
            ici[irp[v] + atomicAdd(&fill[v], 1)] = u;
        }
}

// Directed graphs: combined row v = v's out-arcs, then its in-arcs tagged
// with the top bit; crp = rp + irp; odeg = out-degrees (warp per row).
__global__ void combine_rows_kernel(const int32_t* __restrict__ rp, const int32_t* __restrict__ ci,
                                    const int32_t* __restrict__ irp, const int32_t* __restrict__ ici, int32_t n,
                                    int32_t* __restrict__ crp, int32_t* __restrict__ cci,
                                    int32_t* __restrict__ odeg) {
    const int lane = threadIdx.x & 31;
    const int warp = (blockIdx.x * blockDim.x + threadIdx.x) >> 5;
    const int nwarp = (gridDim.x * blockDim.x) >> 5;
    for (int v = warp; v <= n; v += nwarp) {
        const int base = rp[v] + irp[v];
        if (lane == 0) crp[v] = base;
        if (v == n) continue;
        const int ob = rp[v], od = rp[v + 1] - ob;
        const int ib = irp[v], id = irp[v + 1] - ib;
        if (lane == 0) odeg[v] = od;
        for (int k = lane; k < od; k += 32) cci[base + k] = ci[ob + k];
        for (int k = lane; k < id; k += 32) cci[base + od + k] = (int)((unsigned)ici[ib + k] | 0x80000000u);
    }
}

// Sorted rows: number of distinct neighbours per row (warp per row).
__global__ void unique_count_kernel(const int32_t* __restrict__ rp, const int32_t* __restrict__ ci, int32_t n,
                                    int32_t* __restrict__ cnt) {
    const int lane = threadIdx.x & 31;
    const int warp = (blockIdx.x * blockDim.x + threadIdx.x) >> 5;
    const int nwarp = (gridDim.x * blockDim.x) >> 5;
    for (int v = warp; v < n; v += nwarp) {
        const int b = rp[v], e = rp[v + 1];
        int c = 0;
        for (int k = b + lane; k < e; k += 32) c += (k == b || ci[k] != ci[k - 1]) ? 1 : 0;
        c = warp_sum_i32(c);
        if (lane == 0) cnt[v] = c;
    }
}

__global__ void unique_compact_kernel(const int32_t* __restrict__ rp, const int32_t* __restrict__ ci, int32_t n,
                                      const int32_t* __restrict__ rp2, int32_t* __restrict__ ci2) {
    const int lane = threadIdx.x & 31;
    const int warp = (blockIdx.x * blockDim.x + threadIdx.x) >> 5;
    const int nwarp = (gridDim.x * blockDim.x) >> 5;
    for (int v = warp; v < n; v += nwarp) {
        const int b = rp[v], e = rp[v + 1];
        int out = rp2[v];
        for (int k0 = b; k0 < e; k0 += 32) {
            const int k = k0 + lane;
            const bool keep = k < e && (k == b || ci[k] != ci[k - 1]);
            const unsigned m = __ballot_sync(kFull, keep);
            if (keep) ci2[out + __popc(m & ((1u << lane) - 1u))] = ci[k];
            out += __popc(m);
        }
    }
}

}  // namespace

// Exclusive scan of count int32 values into out[0..count]; out[count] = total.
static sp_status exclusive_scan(const int32_t* d_in, int64_t count, int32_t* d_out, cudaStream_t st) {
    const int64_t nb = (count + kScanBlock - 1) / kScanBlock;
    if (count == 0) {
        SP_CUDA(cudaMemsetAsync(d_out, 0, sizeof(int32_t), st));
        return SP_OK;
    }
    int32_t* sums = nullptr;
    SP_CUDA(cudaMallocAsync((void**)&sums, sizeof(int32_t) * (size_t)(nb + 1), st));
    scan_blocks_kernel<<<(unsigned)nb, kScanBlock, 0, st>>>(d_in, count, d_out, sums);
    cudaError_t e = cudaGetLastError();
    sp_status rc = e == cudaSuccess ? SP_OK : cuda_fail(e, "scan");
    if (rc == SP_OK && nb == 1) {  // one block: its scan is final, its sum is the total
        e = cudaMemcpyAsync(d_out + count, sums, sizeof(int32_t), cudaMemcpyDeviceToDevice, st);
        if (e != cudaSuccess) rc = cuda_fail(e, "scan");
        cudaFreeAsync(sums, st);
        return rc;
    }
    int32_t* offs = nullptr;
    if (rc == SP_OK) {
        e = cudaMallocAsync((void**)&offs, sizeof(int32_t) * (size_t)(nb + 1), st);
        rc = e == cudaSuccess ? exclusive_scan(sums, nb, offs, st) : cuda_fail(e, "scan");
    }
    if (rc == SP_OK) {
        scan_add_kernel<<<(unsigned)nb, kScanBlock, 0, st>>>(d_out, count, offs);
        e = cudaGetLastError();
        if (e == cudaSuccess) e = cudaMemcpyAsync(d_out + count, offs + nb, sizeof(int32_t), cudaMemcpyDeviceToDevice, st);
        if (e != cudaSuccess) rc = cuda_fail(e, "scan");
    }
    if (offs) cudaFreeAsync(offs, st);
    cudaFreeAsync(sums, st);
    return rc;
}

static int current_sms() {
    int dev = 0;
    cudaGetDevice(&dev);
    return device_sm_count(dev);
}

sp_status sort_rows_device(const int32_t* d_rp, int32_t* d_ci, int32_t n, int64_t nnz, cudaStream_t st) {
    if (n == 0 || nnz < 2) return SP_OK;
    const int sms = current_sms();
    int32_t* cnt = nullptr;
    int32_t* lists = nullptr;
    SP_CUDA(cudaMallocAsync((void**)&cnt, sizeof(int32_t) * 4, st));
    cudaError_t e = cudaMallocAsync((void**)&lists, sizeof(int32_t) * 3 * (size_t)n, st);
    if (e != cudaSuccess) { cudaFreeAsync(cnt, st); return cuda_fail(e, "row sort lists"); }
    struct Free {
        std::vector<void*> p;
        cudaStream_t s;
        ~Free() { for (void* x : p) cudaFreeAsync(x, s); }
    } fr{{cnt, lists}, st};
    int32_t* small = lists;
    int32_t* mid = lists + n;
    int32_t* big = lists + 2 * (size_t)n;
    SP_CUDA(cudaMemsetAsync(cnt, 0, sizeof(int32_t) * 4, st));
    classify_rows_kernel<<<sms * 4, 256, 0, st>>>(d_rp, n, cnt, small, mid, big);
    SP_CUDA(cudaGetLastError());
    int32_t h[4] = {0, 0, 0, 0};
    SP_CUDA(cudaMemcpyAsync(h, cnt, sizeof(int32_t) * 4, cudaMemcpyDeviceToHost, st));
    SP_CUDA(cudaStreamSynchronize(st));
    if (h[0] > 0) {
        sort_rows_warp_kernel<<<std::min((h[0] + 7) / 8, sms * 32), 256, 0, st>>>(d_rp, d_ci, small, h[0]);
        SP_CUDA(cudaGetLastError());
    }
    if (h[1] > 0) {
        int2* segs = nullptr;
        SP_CUDA(cudaMallocAsync((void**)&segs, sizeof(int2) * (size_t)h[1], st));
        fr.p.push_back(segs);
        gather_rows_kernel<<<std::min((h[1] + 255) / 256, sms * 4), 256, 0, st>>>(d_rp, mid, h[1], segs);
        sort_segments_block_kernel<<<std::min(h[1], sms * 16), 256, 0, st>>>(d_ci, segs, h[1]);
        SP_CUDA(cudaGetLastError());
    }
    if (h[2] > 0) {
        // long rows: their ranges on the host, 4096-arc pieces sorted in
        // shared memory, then pairwise merges through a compact buffer
        const int nb = h[2];
        int2* d_rows = nullptr;
        SP_CUDA(cudaMallocAsync((void**)&d_rows, sizeof(int2) * (size_t)nb, st));
        fr.p.push_back(d_rows);
        gather_rows_kernel<<<std::min((nb + 255) / 256, sms * 4), 256, 0, st>>>(d_rp, big, nb, d_rows);
        std::vector<int2> rows(nb);
        SP_CUDA(cudaMemcpyAsync(rows.data(), d_rows, sizeof(int2) * (size_t)nb, cudaMemcpyDeviceToHost, st));
        SP_CUDA(cudaStreamSynchronize(st));
        std::sort(rows.begin(), rows.end(), [](int2 x, int2 y) { return x.x < y.x; });
        std::vector<int2> pieces;
        std::vector<int64_t> off_ci(nb), off_tmp(nb);
        std::vector<int32_t> lens(nb);
        int64_t tot = 0;
        int maxlen = 0;
        for (int r = 0; r < nb; ++r) {
            const int len = rows[r].y - rows[r].x;
            for (int p = rows[r].x; p < rows[r].y; p += kSortTile) pieces.push_back(make_int2(p, std::min(p + kSortTile, rows[r].y)));
            off_ci[r] = rows[r].x;
            off_tmp[r] = tot;
            lens[r] = len;
            tot += len;
            maxlen = std::max(maxlen, len);
        }
        int2* d_pieces = nullptr;
        int64_t* d_off = nullptr;
        int32_t* d_lens = nullptr;
        int32_t* tmp = nullptr;
        SP_CUDA(cudaMallocAsync((void**)&d_pieces, sizeof(int2) * pieces.size(), st));
        fr.p.push_back(d_pieces);
        SP_CUDA(cudaMallocAsync((void**)&d_off, sizeof(int64_t) * 2 * (size_t)nb, st));
        fr.p.push_back(d_off);
        SP_CUDA(cudaMallocAsync((void**)&d_lens, sizeof(int32_t) * (size_t)nb, st));
        fr.p.push_back(d_lens);
        SP_CUDA(cudaMallocAsync((void**)&tmp, sizeof(int32_t) * (size_t)tot, st));
        fr.p.push_back(tmp);
        SP_CUDA(cudaMemcpyAsync(d_pieces, pieces.data(), sizeof(int2) * pieces.size(), cudaMemcpyHostToDevice, st));
        SP_CUDA(cudaMemcpyAsync(d_off, off_ci.data(), sizeof(int64_t) * (size_t)nb, cudaMemcpyHostToDevice, st));
        SP_CUDA(cudaMemcpyAsync(d_off + nb, off_tmp.data(), sizeof(int64_t) * (size_t)nb, cudaMemcpyHostToDevice, st));
        SP_CUDA(cudaMemcpyAsync(d_lens, lens.data(), sizeof(int32_t) * (size_t)nb, cudaMemcpyHostToDevice, st));
        sort_segments_block_kernel<<<std::min((int)pieces.size(), sms * 16), 256, 0, st>>>(d_ci, d_pieces,
                                                                                            (int)pieces.size());
        SP_CUDA(cudaGetLastError());
        bool in_ci = true;
        for (int run = kSortTile; run < maxlen; run *= 2) {
            if (in_ci) merge_pass_kernel<<<std::min(nb, sms * 8), 1024, 0, st>>>(d_ci, d_off, tmp, d_off + nb, d_lens, nb, run);
            else merge_pass_kernel<<<std::min(nb, sms * 8), 1024, 0, st>>>(tmp, d_off + nb, d_ci, d_off, d_lens, nb, run);
            SP_CUDA(cudaGetLastError());
            in_ci = !in_ci;
        }
        if (!in_ci)
            for (int r = 0; r < nb; ++r)
                SP_CUDA(cudaMemcpyAsync(d_ci + off_ci[r], tmp + off_tmp[r], sizeof(int32_t) * (size_t)lens[r],
                                        cudaMemcpyDeviceToDevice, st));
    }
    SP_CUDA(cudaStreamSynchronize(st));
    return SP_OK;
}

// Symmetric, deduplicated CSR from an edge list, on the device.  On success
// *d_rp_out / *d_ci_out are cudaMalloc allocations the caller owns.
sp_status csr_from_edges(const int32_t* d_src, const int32_t* d_dst, int64_t m, int32_t n, bool directed,
                         cudaStream_t st, int32_t** d_rp_out, int32_t** d_ci_out, int64_t* nnz_out,
                         std::string* detail) {
    *d_rp_out = nullptr;
    *d_ci_out = nullptr;
    *nnz_out = 0;
    const int sms = current_sms();
    const int egrid = (int)std::max<int64_t>(1, std::min<int64_t>((m + 255) / 256, (int64_t)sms * 8));
    int32_t *deg = nullptr, *rp0 = nullptr, *fill = nullptr, *ci0 = nullptr, *rp = nullptr, *ci = nullptr;
    unsigned long long* bad = nullptr;
    struct Free {
        std::vector<void*> p;
        cudaStream_t s;
        ~Free() { for (void* x : p) if (x) cudaFreeAsync(x, s); }
    } fr{{}, st};
    SP_CUDA(cudaMallocAsync((void**)&deg, sizeof(int32_t) * ((size_t)n + 1), st));
    fr.p.push_back(deg);
    SP_CUDA(cudaMallocAsync((void**)&bad, sizeof(unsigned long long), st));
    fr.p.push_back(bad);
    SP_CUDA(cudaMemsetAsync(deg, 0, sizeof(int32_t) * ((size_t)n + 1), st));
    SP_CUDA(cudaMemsetAsync(bad, 0xFF, sizeof(unsigned long long), st));
    if (m > 0) {
        edge_count_kernel<<<egrid, 256, 0, st>>>(d_src, d_dst, m, n, directed, deg, bad);
        SP_CUDA(cudaGetLastError());
    }
    unsigned long long hbad = 0;
    SP_CUDA(cudaMemcpyAsync(&hbad, bad, sizeof(hbad), cudaMemcpyDeviceToHost, st));
    SP_CUDA(cudaStreamSynchronize(st));
    if (hbad != ~0ull) {
        *detail = "edge " + std::to_string(hbad) + " has an endpoint outside [0, n)";
        return SP_ERR_BAD_GRAPH;
    }
    SP_CUDA(cudaMallocAsync((void**)&rp0, sizeof(int32_t) * ((size_t)n + 1), st));
    fr.p.push_back(rp0);
    sp_status rc = exclusive_scan(deg, n, rp0, st);
    if (rc != SP_OK) return rc;
    int32_t arcs = 0;
    SP_CUDA(cudaMemcpyAsync(&arcs, rp0 + n, sizeof(int32_t), cudaMemcpyDeviceToHost, st));
    SP_CUDA(cudaStreamSynchronize(st));
    SP_CUDA(cudaMallocAsync((void**)&fill, sizeof(int32_t) * ((size_t)n + 1), st));
    fr.p.push_back(fill);
    SP_CUDA(cudaMallocAsync((void**)&ci0, sizeof(int32_t) * (size_t)std::max(arcs, 1), st));
    fr.p.push_back(ci0);
    SP_CUDA(cudaMemsetAsync(fill, 0, sizeof(int32_t) * ((size_t)n + 1), st));
    if (m > 0) {
        edge_scatter_kernel<<<egrid, 256, 0, st>>>(d_src, d_dst, m, directed, rp0, fill, ci0);
        SP_CUDA(cudaGetLastError());
    }
    rc = sort_rows_device(rp0, ci0, n, arcs, st);
    if (rc != SP_OK) return rc;
    const int wgrid = std::max(1, std::min((n + 7) / 8, sms * 16));
    if (n > 0) {
        unique_count_kernel<<<wgrid, 256, 0, st>>>(rp0, ci0, n, deg);
        SP_CUDA(cudaGetLastError());
    }
    // the final arrays outlive the call (the graph object frees them with cudaFree)
    SP_CUDA(cudaMalloc((void**)&rp, sizeof(int32_t) * ((size_t)n + 1)));
    rc = exclusive_scan(deg, n, rp, st);
    if (rc != SP_OK) { cudaFree(rp); return rc; }
    int32_t nnz = 0;
    cudaError_t e = cudaMemcpyAsync(&nnz, rp + n, sizeof(int32_t), cudaMemcpyDeviceToHost, st);
    if (e == cudaSuccess) e = cudaStreamSynchronize(st);
    if (e != cudaSuccess) { cudaFree(rp); return cuda_fail(e, "edge-list CSR"); }
    if (cudaMalloc((void**)&ci, sizeof(int32_t) * (size_t)std::max(nnz, 1)) != cudaSuccess) {
        cudaGetLastError();
        cudaFree(rp);
        return fail(SP_ERR_OOM, "edge-list CSR");
    }
    if (n > 0) unique_compact_kernel<<<wgrid, 256, 0, st>>>(rp0, ci0, n, rp, ci);
    e = cudaGetLastError();
    if (e == cudaSuccess) e = cudaStreamSynchronize(st);
    if (e != cudaSuccess) {
        cudaFree(rp);
        cudaFree(ci);
        return cuda_fail(e, "edge-list CSR");
    }
    *d_rp_out = rp;
    *d_ci_out = ci;
    *nnz_out = nnz;
    return SP_OK;
}

// Directed graphs: the combined rows the kernels read (out-arcs, then in-arcs
// tagged with the top bit, in increasing source id) and the out-degrees, built
// on the device from the out-arc CSR.  The three outputs are cudaMalloc
// allocations the caller owns.  2 nnz must be below 2^31.
sp_status combined_rows(const int32_t* d_rp, const int32_t* d_ci, int32_t n, int64_t nnz, cudaStream_t st,
                        int32_t** d_crp, int32_t** d_cci, int32_t** d_odeg) {
    *d_crp = *d_cci = *d_odeg = nullptr;
    if (2 * nnz >= (int64_t)INT32_MAX) return fail(SP_ERR_TOO_LARGE, "directed graphs need 2 nnz below 2^31");
    const int sms = current_sms();
    int32_t *indeg = nullptr, *irp = nullptr, *fill = nullptr, *ici = nullptr;
    struct Free {
        std::vector<void*> p;
        cudaStream_t s;
        ~Free() { for (void* x : p) if (x) cudaFreeAsync(x, s); }
    } fr{{}, st};
    SP_CUDA(cudaMallocAsync((void**)&indeg, sizeof(int32_t) * ((size_t)n + 1), st));
    fr.p.push_back(indeg);
    SP_CUDA(cudaMallocAsync((void**)&irp, sizeof(int32_t) * ((size_t)n + 1), st));
    fr.p.push_back(irp);
    SP_CUDA(cudaMallocAsync((void**)&fill, sizeof(int32_t) * ((size_t)n + 1), st));
    fr.p.push_back(fill);
    SP_CUDA(cudaMallocAsync((void**)&ici, sizeof(int32_t) * (size_t)std::max<int64_t>(nnz, 1), st));
    fr.p.push_back(ici);
    SP_CUDA(cudaMemsetAsync(indeg, 0, sizeof(int32_t) * ((size_t)n + 1), st));
    SP_CUDA(cudaMemsetAsync(fill, 0, sizeof(int32_t) * ((size_t)n + 1), st));
    const int egrid = (int)std::max<int64_t>(1, std::min<int64_t>((nnz + 255) / 256, (int64_t)sms * 8));
    const int wgrid = std::max(1, std::min((n + 8) / 8, sms * 16));
    if (nnz > 0) in_count_kernel<<<egrid, 256, 0, st>>>(d_ci, nnz, indeg);
    SP_CUDA(cudaGetLastError());
    sp_status rc = exclusive_scan(indeg, n, irp, st);
    if (rc != SP_OK) return rc;
    if (n > 0) in_scatter_kernel<<<wgrid, 256, 0, st>>>(d_rp, d_ci, n, irp, fill, ici);
    SP_CUDA(cudaGetLastError());
    rc = sort_rows_device(irp, ici, n, nnz, st);
    if (rc != SP_OK) return rc;
    int32_t *crp = nullptr, *cci = nullptr, *odeg = nullptr;
    if (cudaMalloc((void**)&crp, sizeof(int32_t) * ((size_t)n + 1)) != cudaSuccess ||
        cudaMalloc((void**)&cci, sizeof(int32_t) * (size_t)std::max<int64_t>(2 * nnz, 1)) != cudaSuccess ||
        cudaMalloc((void**)&odeg, sizeof(int32_t) * (size_t)std::max<int32_t>(n, 1)) != cudaSuccess) {
        cudaGetLastError();
        cudaFree(crp);
        cudaFree(cci);
        cudaFree(odeg);
        return fail(SP_ERR_OOM, "directed graph rows");
    }
    combine_rows_kernel<<<wgrid, 256, 0, st>>>(d_rp, d_ci, irp, ici, n, crp, cci, odeg);
    cudaError_t e = cudaGetLastError();
    if (e == cudaSuccess) e = cudaStreamSynchronize(st);
    if (e != cudaSuccess) {
        cudaFree(crp);
        cudaFree(cci);
        cudaFree(odeg);
        return cuda_fail(e, "directed graph rows");
    }
    *d_crp = crp;
    *d_cci = cci;
    *d_odeg = odeg;
    return SP_OK;
}

}  // namespace sp
