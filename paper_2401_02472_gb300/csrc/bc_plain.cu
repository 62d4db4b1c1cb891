// Host launcher of the plain form (kernel in bc_plain_kernel.cuh).
#include <algorithm>
#include <climits>
#include <cstdio>
#include <cstring>
#include <vector>
#include <string>

#include "bc_plain_kernel.cuh"

namespace sp {

template <typename SigT, typename ThT>
static const void* plain_fn(bool rec, bool dir) {
    if (dir)
        return rec ? reinterpret_cast<const void*>(&plain_kernel<SigT, ThT, true, true>)
                   : reinterpret_cast<const void*>(&plain_kernel<SigT, ThT, false, true>);
    return rec ? reinterpret_cast<const void*>(&plain_kernel<SigT, ThT, true, false>)
               : reinterpret_cast<const void*>(&plain_kernel<SigT, ThT, false, false>);
}

sp_status run_plain(const PlainLaunch& L, LaunchResult* result) {
    const Graph* g = L.g;
    const int64_t n = g->n;
    cudaStream_t st = L.stream;
    Tiers tiers{16, 4096, 4096};
    const bool dir = g->directed;
    auto pick = [&](bool rec) {
        if (L.sigma_float) return L.theta_f32 ? plain_fn<double, float>(rec, dir) : plain_fn<double, double>(rec, dir);
        return L.theta_f32 ? plain_fn<unsigned long long, float>(rec, dir)
                           : plain_fn<unsigned long long, double>(rec, dir);
    };
    const void* fn = pick(false);

    int dev = g->device;
    int per_sm = 0;
    SP_CUDA(cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, fn, kPlainThreads, 0));
    if (per_sm < 1) return fail(SP_ERR_CUDA, "plain kernel cannot be resident");
    int grid = per_sm * device_sm_count(dev);
    if (L.max_ctas > 0 && L.max_ctas < grid) grid = L.max_ctas;
    // Groups: `group_blocks` blocks each (0 = one group of every block), no
    // more groups than sources (blocks beyond them are not launched: narrow
    // levels gain nothing from more blocks but barrier cost); a
    // fault-injection run keeps one group so that the skipped barrier is a
    // real multi-block wait.
    int gblocks = L.group_blocks > 0 ? std::min(L.group_blocks, grid) : grid;
    if (L.debug_flags & SP_DEBUG_SKIP_BARRIER) gblocks = grid;
    int ngroups = std::max(1, std::min(grid / gblocks, std::max(1, L.nsrc)));
    grid = ngroups * gblocks;

    // Vertex records instead of arrays when several groups' state (level,
    // path count, theta, partial BC: 28 bytes a vertex) is more than twice L2:
    // there each access misses, and a record puts a vertex's level test and
    // its path count or theta in one sector.
    int l2 = 0;
    cudaDeviceGetAttribute(&l2, cudaDevAttrL2CacheSize, dev);
    bool rec = ngroups > 1 && L.mode == PlainMode::BC && (double)ngroups * (double)n * 28.0 > 2.0 * (double)l2;
    if (L.debug_flags & SP_DEBUG_PLAIN_RECORDS) rec = true;
    if (L.debug_flags & SP_DEBUG_PLAIN_ARRAYS) rec = false;
    if (L.d_sq != nullptr) rec = false;  // the squared dependencies need the partial arrays
    if (rec) {
        int per_sm_rec = 0;
        SP_CUDA(cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm_rec, pick(true), kPlainThreads, 0));
        if (per_sm_rec < per_sm) rec = false;  // keep the grid co-resident
        else fn = pick(true);
    }

    // Workspace: one copy of the per-source arrays per group.
    const int64_t lcap = L.level_cap > 0 ? std::min<int64_t>(L.level_cap, n + 2)
                                         : (ngroups == 1 ? n + 2 : std::min<int64_t>(n + 2, 65536));
    const int64_t hcap = g->knnz() / tiers.t_hub + 2;
    const int64_t segcap = g->knnz() / tiers.seg + hcap + 2;
    const PlainLayout lay = plain_layout(n, lcap, hcap, segcap, ngroups, grid, ngroups > 1 && L.mode == PlainMode::BC, rec,
                                         L.d_sq != nullptr);
    const size_t bytes = lay.bytes;
    char* ws = nullptr;
    cudaError_t ce = workspace_alloc((void**)&ws, bytes, st);
    if (ce != cudaSuccess) {
        cudaGetLastError();
        return fail(SP_ERR_OOM, "workspace allocation (plain form, " + std::to_string(bytes >> 20) + " MiB)");
    }
    ce = cudaMemsetAsync(ws, 0, lay.zero_end, st);
    if (ce != cudaSuccess) { cudaFreeAsync(ws, st); return cuda_fail(ce, "cudaMemsetAsync"); }

    PlainArgs a{};
    a.rp = g->krp();
    a.ci = g->kci();
    a.directed = g->directed;
    a.odeg = g->d_odeg;
    a.n = (int32_t)n;
    a.sources = L.d_sources;
    a.nsrc = L.nsrc;
    a.bc = L.d_bc;
    plain_bind(a, ws, lay);
    a.sq = L.mode == PlainMode::BC ? L.d_sq : nullptr;
    a.gblocks = gblocks;
    a.ngroups = ngroups;
    a.hcap = (int32_t)hcap;
    a.segcap = (int32_t)segcap;
    a.lcap = (int32_t)lcap;
    a.pre_err = L.async.pre_err;
    a.gate = L.async.gate;
    a.dist_out = L.d_dist;
    a.mant_out = L.d_mant;
    a.exp_out = L.d_exp;
    a.mode = (int)L.mode;
    a.debug_flags = L.debug_flags;
    a.timeout_ns = L.timeout_ns;
    a.t_thread = tiers.t_thread;
    a.t_hub = tiers.t_hub;
    a.seg = tiers.seg;
    a.bu_den = L.bottom_up_den;
    a.centre_bound = sigma_centre_bound(L.sigma_float, L.theta_f32, L.mode);
    cudaMemsetAsync(a.trace, 0, sizeof(int) * 8 * (size_t)grid * (kPlainThreads / 32), st);

    void* args[] = {&a};
    auto launch = [&]() -> cudaError_t {
        cudaError_t e = cudaLaunchCooperativeKernel(fn, dim3(grid), dim3(kPlainThreads), args, 0, st);
        if (e == cudaSuccess && ngroups > 1 && L.mode == PlainMode::BC) {
            int rgrid = (int)std::min<int64_t>((n + 255) / 256, (int64_t)device_sm_count(dev) * 8);
            const double* part = rec ? reinterpret_cast<const double*>(a.lvl) + 1 : a.bcpart;
            sum_group_partials_kernel<<<std::max(rgrid, 1), 256, 0, st>>>(part, ngroups, n, rec ? 4 : 1, L.d_bc,
                                                                          a.gate);
            if (a.sq != nullptr)
                sum_group_partials_kernel<<<std::max(rgrid, 1), 256, 0, st>>>(a.sqpart, ngroups, n, 1, a.sq, a.gate);
            e = cudaGetLastError();
        }
        return e;
    };
    if (L.async.flags != nullptr) {  // enqueue only: the finish step moves the error word on
        ce = launch();
        if (ce != cudaSuccess) {
            cudaFreeAsync(ws, st);
            return cuda_fail(ce, "plain-form launch");
        }
        sp_status frc = enqueue_finish(a.ctl, L.async, st);
        cudaFreeAsync(ws, st);
        result->launches = ngroups > 1 && L.mode == PlainMode::BC ? 3 : 2;
        result->lcap = lcap;
        result->grid = grid;
        result->groups = ngroups;
        return frc;
    }
    cudaEvent_t ev0, ev1;
    cudaEventCreate(&ev0);
    cudaEventCreate(&ev1);
    cudaEventRecord(ev0, st);
    ce = launch();
    cudaEventRecord(ev1, st);
    if (ce != cudaSuccess) {
        cudaFreeAsync(ws, st);
        cudaEventDestroy(ev0);
        cudaEventDestroy(ev1);
        return cuda_fail(ce, "plain-form launch");
    }
    static thread_local Ctl h;
    std::memset(&h, 0, sizeof(h));
    ce = cudaMemcpyAsync(&h, ws + lay.ctl, sizeof(Ctl), cudaMemcpyDeviceToHost, st);
    if (ce == cudaSuccess) ce = cudaStreamSynchronize(st);
    if (ce != cudaSuccess) {
        cudaFreeAsync(ws, st);
        return cuda_fail(ce, "reading the plain-form result");
    }
    result->err = h.err;
    result->levels = h.max_levels;
    result->traversed_arcs = h.traversed_arcs;
    result->reached = h.reached;
    result->entries = h.reached;
    result->scanned_arcs = h.scanned_arcs;
    result->dag_arcs = h.dag_arcs;
    result->recentred = h.recentred;
    result->lcap = lcap;
    result->grid = grid;
    result->groups = ngroups;
    float ms = 0.0f;
    if (cudaEventElapsedTime(&ms, ev0, ev1) == cudaSuccess) result->kernel_ms = ms;
    cudaEventDestroy(ev0);
    cudaEventDestroy(ev1);
    result->launches = ngroups > 1 && L.mode == PlainMode::BC ? 2 : 1;
    if (h.err == SP_ERR_TIMEOUT) result->diag = barrier_diagnostic(h, grid);
#ifdef SP_TRACE
    if (h.err == SP_ERR_TIMEOUT) {
        std::vector<int> tr(8 * (size_t)grid * (kPlainThreads / 32));
        cudaMemcpy(tr.data(), ws + lay.trace, sizeof(int) * tr.size(), cudaMemcpyDeviceToHost);
        int lo = INT32_MAX;
        for (int b = 0; b < grid; ++b) lo = std::min(lo, h.block_phase[b]);
        for (int b = 0; b < grid; ++b) {
            if (h.block_phase[b] != lo) continue;
            for (int w = 0; w < kPlainThreads / 32; ++w) {
                const int* t = &tr[8 * ((size_t)b * (kPlainThreads / 32) + w)];
                fprintf(stderr, "trace block %d warp %d: phase %d item %d total %d nseg %d qb %d qe %d d %d n %d\n", b, w,
                        t[0], t[1], t[2], t[3], t[4], t[5], t[6], t[7]);
            }
        }
    }
#endif
    cudaFreeAsync(ws, st);
    return SP_OK;
}

}  // namespace sp
