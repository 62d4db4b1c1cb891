// PageRank over a resident graph: the pull form of the paper's reduction
// listing for PageRank (Section 3.3, the OpenACC listing over the reverse
// CSR): every iteration gives each vertex v
//
//     PR'(v) = (1 - d) / N + d * sum over in-neighbours u of PR(u) / outdeg(u)
//
// and adds |PR'(v) - PR(v)| to the iteration's change; the loop stops after
// the first iteration whose change is at most `tol` (never when tol < 0) or
// after `max_iter` iterations.  PR starts at 1 / N; a vertex without out-arcs
// passes nothing on.
//
// One persistent cooperative launch runs every iteration.  Per iteration:
//   items   rows of 32 consecutive vertices (a lane walks a row of at most 16
//           arcs in CSR order, the warp walks longer ones), and segments of
//           `seg` arcs of the rows longer than `seg` (hubs), whose partial
//           sums the last segment to finish adds in segment order; warps take
//           items from a shared counter.  Each vertex writes PR', PR' /
//           outdeg (what its out-neighbours read next) and |PR' - PR|.
//   change  after a grid barrier each block sums a fixed slice of the
//           changes in a fixed order; after a second barrier every block adds
//           the blocks' sums in block order, so all blocks take the same
//           stop decision and the result is the same bit for bit run to run.
// Pull sums, no floating-point atomics.  Directed graphs read the combined
// rows (out-arcs, then tagged in-arcs) and sum over the in-arcs only.
#include <cuda_runtime.h>

#include <algorithm>
#include <cstring>
#include <mutex>
#include <string>
#include <vector>

#include "common.cuh"
#include "internal.h"

namespace sp {
namespace {

constexpr int kPrThreads = 512;
constexpr int kPrLane = 16;  // rows of at most this many arcs are walked by one lane

struct PrArgs {
    const int32_t* rp;
    const int32_t* ci;
    const int32_t* odeg;  // out-degrees (directed graphs); null: the row length
    int32_t n;
    int directed;
    const int32_t* hubs;      // [nhubs] rows longer than seg
    const int32_t* hub_seg0;  // [nhubs + 1] first segment of each hub
    int32_t nhubs;
    int32_t nseg;
    int32_t seg;
    double damping, tol;
    int32_t max_iter;
    double* pr0;         // the caller's output (PR of even iterations)
    double* pr1;         // PR of odd iterations
    double* contrib0;    // PR / outdeg of the ranks in pr0
    double* contrib1;
    double* change;      // [n] |PR' - PR| of the iteration
    double* seg_part;    // [nseg] hub segment partial sums
    unsigned* hub_done;  // [nhubs] segments finished, cumulative over iterations
    double* part;        // [gridDim.x] block sums of the change
    Ctl* ctl;
    const int* pre_err;  // asynchronous calls: unused (no sources), kept for the common skip rule
    unsigned long long timeout_ns;
    int32_t* iters_out;  // device
    double* change_out;  // device
};

__device__ __forceinline__ bool is_hub(const PrArgs& a, int deg) { return deg > a.seg; }

__device__ __forceinline__ double inv_out(const PrArgs& a, int v, int row_len) {
    const int od = a.odeg != nullptr ? __ldg(&a.odeg[v]) : row_len;
    return od > 0 ? 1.0 / (double)od : 0.0;
}

// New rank of v from its pull sum; writes PR', PR' / outdeg and the change.
__device__ __forceinline__ void settle(const PrArgs& a, int v, int row_len, double sum, const double* pr_cur,
                                      double* pr_nxt, double* contrib_nxt) {
    const double val = (1.0 - a.damping) / (double)a.n + a.damping * sum;
    pr_nxt[v] = val;
    const int od = a.odeg != nullptr ? __ldg(&a.odeg[v]) : row_len;
    contrib_nxt[v] = od > 0 ? val / (double)od : 0.0;
    a.change[v] = fabs(val - __ldcg(&pr_cur[v]));
}

// Rows [32c, 32c + 32) that are not hubs.
__device__ void rows_item(const PrArgs& a, int c, const double* contrib, const double* pr_cur, double* pr_nxt,
                          double* contrib_nxt) {
    const int lane = lane_id();
    const int v = c * 32 + lane;
    int beg = 0, deg = 0;
    if (v < a.n) {
        beg = __ldg(&a.rp[v]);
        deg = __ldg(&a.rp[v + 1]) - beg;
    }
    double sum = 0.0;
    const bool mine = v < a.n && deg <= kPrLane;
    if (mine) {
        for (int k = 0; k < deg; ++k) {
            const int raw = __ldg(&a.ci[beg + k]);
            if (arc_in(raw, a.directed)) sum += __ldcg(&contrib[arc_vertex(raw)]);
        }
    }
    unsigned wide = __ballot_sync(kFull, v < a.n && deg > kPrLane && !is_hub(a, deg));
    while (wide) {
        const int j = __ffs(wide) - 1;
        wide &= wide - 1;
        const int bj = __shfl_sync(kFull, beg, j), dj = __shfl_sync(kFull, deg, j);
        double p = 0.0;
        for (int k = lane; k < dj; k += kWarp) {
            const int raw = __ldg(&a.ci[bj + k]);
            if (arc_in(raw, a.directed)) p += __ldcg(&contrib[arc_vertex(raw)]);
        }
        p = warp_sum_f64(p);
        if (lane == j) sum = p;
    }
    if (v < a.n && !is_hub(a, deg)) settle(a, v, deg, sum, pr_cur, pr_nxt, contrib_nxt);
}

// Segment g of the hub rows; the last segment of a hub to finish settles it.
__device__ void hub_item(const PrArgs& a, int g, int iter, const double* contrib, const double* pr_cur,
                         double* pr_nxt, double* contrib_nxt) {
    const int lane = lane_id();
    int lo = 0, hi = a.nhubs;  // the hub whose segments hold g: hub_seg0[h] <= g < hub_seg0[h + 1]
    while (hi - lo > 1) {
        const int mid = (lo + hi) >> 1;
        if (__ldg(&a.hub_seg0[mid]) <= g) lo = mid; else hi = mid;
    }
    const int h = lo;
    const int v = __ldg(&a.hubs[h]);
    const int s0 = __ldg(&a.hub_seg0[h]), ns = __ldg(&a.hub_seg0[h + 1]) - s0;
    const int rb = __ldg(&a.rp[v]), re = __ldg(&a.rp[v + 1]);
    const int b = rb + (g - s0) * a.seg, e = min(re, b + a.seg);
    double p = 0.0;
    for (int k = b + lane; k < e; k += kWarp) {
        const int raw = __ldg(&a.ci[k]);
        if (arc_in(raw, a.directed)) p += __ldcg(&contrib[arc_vertex(raw)]);
    }
    p = warp_sum_f64(p);
    unsigned old = 0;
    if (lane == 0) {
        a.seg_part[g] = p;
        __threadfence();
        old = atomicAdd(&a.hub_done[h], 1u);
    }
    old = __shfl_sync(kFull, old, 0);
    if (old != (unsigned)(iter + 1) * (unsigned)ns - 1u) return;
    __threadfence();
    double t = 0.0;
    for (int q = lane; q < ns; q += kWarp) t += __ldcg(&a.seg_part[s0 + q]);
    t = warp_sum_f64(t);
    if (lane == 0) settle(a, v, re - rb, t, pr_cur, pr_nxt, contrib_nxt);
}

#ifndef SP_PR_PER_SM
#define SP_PR_PER_SM 2  // resident blocks per SM the registers are sized for
#endif
__global__ void __launch_bounds__(kPrThreads, SP_PR_PER_SM) pagerank_kernel(PrArgs a) {
    if (a.pre_err != nullptr && ld_volatile(a.pre_err) != 0) return;
    Ctl* ctl = a.ctl;
    const int tid = blockIdx.x * blockDim.x + threadIdx.x;
    const int nthr = gridDim.x * blockDim.x;
    const int nwarps = nthr / kWarp, gwarp = tid / kWarp;
    int phase = 0, snap = 0;
    auto sync = [&]() -> bool {
        const bool ok = grid_sync(ctl, gridDim.x, a.timeout_ns, phase++, false, &snap);
        if (tid == 0) ctl->work[(phase + 2) & 3] = 0u;
        return ok;
    };
    const int n = a.n;
    for (int v = tid; v < n; v += nthr) {
        const double p = 1.0 / (double)n;
        a.pr0[v] = p;
        const int od = a.odeg != nullptr ? __ldg(&a.odeg[v]) : __ldg(&a.rp[v + 1]) - __ldg(&a.rp[v]);
        a.contrib0[v] = od > 0 ? p / (double)od : 0.0;
    }
    int iter = 0;
    double total = 0.0;
    if (!sync()) return;
    const int nrows = (n + 31) / 32;
    const int items = nrows + a.nseg;
    while (iter < a.max_iter) {
        const bool odd = iter & 1;
        const double* pr_cur = odd ? a.pr1 : a.pr0;
        double* pr_nxt = odd ? a.pr0 : a.pr1;
        const double* contrib = odd ? a.contrib1 : a.contrib0;
        double* contrib_nxt = odd ? a.contrib0 : a.contrib1;
        for (int item = gwarp; item < items;) {
            if (item < a.nseg) hub_item(a, item, iter, contrib, pr_cur, pr_nxt, contrib_nxt);
            else rows_item(a, item - a.nseg, contrib, pr_cur, pr_nxt, contrib_nxt);
            if (nwarps >= items) break;
            int next = 0;
            if (lane_id() == 0) next = nwarps + (int)atomicAdd(&ctl->work[phase & 3], 1u);
            item = __shfl_sync(kFull, next, 0);
        }
        if (!sync()) return;
        // this block's fixed slice of the changes, in a fixed order
        {
            __shared__ double s_w[kPrThreads / kWarp];
            const int per = (n + gridDim.x - 1) / gridDim.x;
            const int lo = blockIdx.x * per, hi = min(n, lo + per);
            double x = 0.0;
            for (int v = lo + threadIdx.x; v < hi; v += blockDim.x) x += __ldcg(&a.change[v]);
            x = warp_sum_f64(x);
            if (lane_id() == 0) s_w[threadIdx.x / kWarp] = x;
            __syncthreads();
            if (threadIdx.x == 0) {
                double b = 0.0;
                for (int w = 0; w < (int)(blockDim.x / kWarp); ++w) b += s_w[w];
                a.part[blockIdx.x] = b;
            }
        }
        if (!sync()) return;
        __shared__ double s_total;
        if (threadIdx.x == 0) {
            double t = 0.0;
            for (int b = 0; b < (int)gridDim.x; ++b) t += __ldcg(&a.part[b]);
            s_total = t;
        }
        __syncthreads();
        total = s_total;
        ++iter;
        if (a.tol >= 0.0 && total <= a.tol) break;
    }
    // the ranks of an odd number of iterations sit in pr1: move them out
    if (iter & 1)
        for (int v = tid; v < n; v += nthr) a.pr0[v] = __ldcg(&a.pr1[v]);
    if (tid == 0) {
        *a.iters_out = iter;
        *a.change_out = total;
    }
}

// Hub rows of a graph (rows longer than the segment), found once per graph.
struct PrPlan {
    int32_t* hubs = nullptr;
    int32_t* hub_seg0 = nullptr;
    int32_t nhubs = 0, nseg = 0;
};
std::mutex g_plan_mu;

sp_status pr_plan(Graph* g, int seg, cudaStream_t st, PrPlan* out) {
    std::vector<int32_t> rp((size_t)g->n + 1);
    SP_CUDA(cudaMemcpyAsync(rp.data(), g->krp(), sizeof(int32_t) * rp.size(), cudaMemcpyDeviceToHost, st));
    SP_CUDA(cudaStreamSynchronize(st));
    std::vector<int32_t> hubs, seg0{0};
    for (int32_t v = 0; v < g->n; ++v) {
        const int64_t deg = rp[v + 1] - rp[v];
        if (deg > seg) {
            hubs.push_back(v);
            seg0.push_back(seg0.back() + (int32_t)((deg + seg - 1) / seg));
        }
    }
    out->nhubs = (int32_t)hubs.size();
    out->nseg = seg0.back();
    SP_CUDA(cudaMalloc((void**)&out->hubs, sizeof(int32_t) * std::max<size_t>(hubs.size(), 1)));
    SP_CUDA(cudaMalloc((void**)&out->hub_seg0, sizeof(int32_t) * seg0.size()));
    if (!hubs.empty())
        SP_CUDA(cudaMemcpyAsync(out->hubs, hubs.data(), sizeof(int32_t) * hubs.size(), cudaMemcpyHostToDevice, st));
    SP_CUDA(cudaMemcpyAsync(out->hub_seg0, seg0.data(), sizeof(int32_t) * seg0.size(), cudaMemcpyHostToDevice, st));
    SP_CUDA(cudaStreamSynchronize(st));
    return SP_OK;
}

}  // namespace

constexpr int kPrSeg = 2048;  // arcs per hub segment

void destroy_pr_plan(Graph* g) {
    PrPlan* p = static_cast<PrPlan*>(g->pr_plan);
    if (!p) return;
    if (p->hubs) cudaFree(p->hubs);
    if (p->hub_seg0) cudaFree(p->hub_seg0);
    delete p;
    g->pr_plan = nullptr;
}

sp_status run_pagerank(const PrLaunch& L, PrResult* result) {
    Graph* g = L.g;
    const int64_t n = g->n;
    cudaStream_t st = L.stream;
    PrPlan plan;
    {
        std::lock_guard<std::mutex> lk(g_plan_mu);
        if (!g->pr_plan) {
            PrPlan* p = new PrPlan();
            sp_status rc = pr_plan(g, kPrSeg, st, p);
            if (rc != SP_OK) {
                if (p->hubs) cudaFree(p->hubs);
                if (p->hub_seg0) cudaFree(p->hub_seg0);
                delete p;
                return rc;
            }
            g->pr_plan = p;
        }
        plan = *static_cast<PrPlan*>(g->pr_plan);
    }
    int per_sm = 0;
    SP_CUDA(cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, (const void*)&pagerank_kernel, kPrThreads, 0));
    if (per_sm < 1) return fail(SP_ERR_CUDA, "pagerank kernel cannot be resident");
    int grid = per_sm * device_sm_count(g->device);
    if (L.max_ctas > 0 && L.max_ctas < grid) grid = L.max_ctas;

    size_t bytes = 0;
    auto take = [&](size_t b) { size_t o = bytes; bytes += (b + 255) & ~(size_t)255; return o; };
    const size_t o_ctl = take(sizeof(Ctl));
    const size_t o_done = take(sizeof(unsigned) * (size_t)std::max(plan.nhubs, 1));
    const size_t o_res = take(sizeof(double) + sizeof(int32_t));
    const size_t zero_end = bytes;
    const size_t o_pr1 = take(sizeof(double) * (size_t)n);
    const size_t o_c0 = take(sizeof(double) * (size_t)n);
    const size_t o_c1 = take(sizeof(double) * (size_t)n);
    const size_t o_chg = take(sizeof(double) * (size_t)n);
    const size_t o_seg = take(sizeof(double) * (size_t)std::max(plan.nseg, 1));
    const size_t o_part = take(sizeof(double) * (size_t)grid);
    char* ws = nullptr;
    if (workspace_alloc((void**)&ws, bytes, st) != cudaSuccess) {
        cudaGetLastError();
        return fail(SP_ERR_OOM, "workspace allocation (pagerank)");
    }
    cudaError_t ce = cudaMemsetAsync(ws, 0, zero_end, st);
    if (ce != cudaSuccess) {
        cudaFreeAsync(ws, st);
        return cuda_fail(ce, "cudaMemsetAsync");
    }
    PrArgs a{};
    a.rp = g->krp();
    a.ci = g->kci();
    a.odeg = g->d_odeg;
    a.n = (int32_t)n;
    a.directed = g->directed;
    a.hubs = plan.hubs;
    a.hub_seg0 = plan.hub_seg0;
    a.nhubs = plan.nhubs;
    a.nseg = plan.nseg;
    a.seg = kPrSeg;
    a.damping = L.damping;
    a.tol = L.tol;
    a.max_iter = L.max_iter;
    a.pr0 = L.d_pr;
    a.pr1 = reinterpret_cast<double*>(ws + o_pr1);
    a.contrib0 = reinterpret_cast<double*>(ws + o_c0);
    a.contrib1 = reinterpret_cast<double*>(ws + o_c1);
    a.change = reinterpret_cast<double*>(ws + o_chg);
    a.seg_part = reinterpret_cast<double*>(ws + o_seg);
    a.hub_done = reinterpret_cast<unsigned*>(ws + o_done);
    a.part = reinterpret_cast<double*>(ws + o_part);
    a.ctl = reinterpret_cast<Ctl*>(ws + o_ctl);
    a.pre_err = nullptr;
    a.timeout_ns = L.timeout_ns;
    a.change_out = reinterpret_cast<double*>(ws + o_res);
    a.iters_out = reinterpret_cast<int32_t*>(ws + o_res + sizeof(double));
    void* args[] = {&a};
    if (L.async.flags != nullptr) {  // enqueue only: the finish step latches an error
        ce = cudaLaunchCooperativeKernel((const void*)&pagerank_kernel, dim3(grid), dim3(kPrThreads), args, 0, st);
        if (ce != cudaSuccess) {
            cudaFreeAsync(ws, st);
            return cuda_fail(ce, "pagerank launch");
        }
        sp_status rc = enqueue_finish(a.ctl, L.async, st);
        cudaFreeAsync(ws, st);
        result->launches = 2;
        return rc;
    }
    cudaEvent_t ev0, ev1;
    cudaEventCreate(&ev0);
    cudaEventCreate(&ev1);
    cudaEventRecord(ev0, st);
    ce = cudaLaunchCooperativeKernel((const void*)&pagerank_kernel, dim3(grid), dim3(kPrThreads), args, 0, st);
    cudaEventRecord(ev1, st);
    struct {
        double change;
        int32_t iters;
    } res{0.0, 0};
    static thread_local Ctl h;
    std::memset(&h, 0, sizeof(h));
    if (ce == cudaSuccess) ce = cudaMemcpyAsync(&h, ws + o_ctl, sizeof(Ctl), cudaMemcpyDeviceToHost, st);
    if (ce == cudaSuccess) ce = cudaMemcpyAsync(&res.change, ws + o_res, sizeof(double), cudaMemcpyDeviceToHost, st);
    if (ce == cudaSuccess)
        ce = cudaMemcpyAsync(&res.iters, ws + o_res + sizeof(double), sizeof(int32_t), cudaMemcpyDeviceToHost, st);
    cudaFreeAsync(ws, st);
    if (ce == cudaSuccess) ce = cudaStreamSynchronize(st);
    float ms = 0.0f;
    if (ce == cudaSuccess && cudaEventElapsedTime(&ms, ev0, ev1) == cudaSuccess) result->kernel_ms = ms;
    cudaEventDestroy(ev0);
    cudaEventDestroy(ev1);
    if (ce != cudaSuccess) return cuda_fail(ce, "pagerank");
    result->err = h.err;
    result->iterations = res.iters;
    result->change = res.change;
    result->launches = 1;
    result->grid = grid;
    if (h.err == SP_ERR_TIMEOUT) result->diag = barrier_diagnostic(h, grid);
    return SP_OK;
}

}  // namespace sp
